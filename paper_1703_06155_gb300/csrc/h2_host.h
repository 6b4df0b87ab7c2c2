// Host-side data structures of libh2: cluster tree, block partition, the H^2
// representation (FP64, tree order) and the per-context device state.
#pragma once
#include <chrono>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/h2.h"
#include "h2_kernels.h"

namespace h2 {

using cplx = std::complex<double>;
using Pair = std::pair<int, int>;

inline int64_t pkey(int a, int b) { return ((int64_t)a << 32) | (uint32_t)b; }

// Complete binary cluster tree (Sec. II): level l has 2^l clusters; cluster c
// covers tree positions [start, start+size); children are 2c, 2c+1.
struct Tree {
  int64_t N = 0;
  int L = 0;
  std::vector<int64_t> perm;                 // tree position -> global index
  std::vector<std::vector<int64_t>> start, size;
  std::vector<std::vector<double>> centre;   // 3 per cluster
  std::vector<std::vector<double>> radius;
};

// Admissible / inadmissible same-level pairs (eq. 1), sorted per level.
struct Partition {
  std::vector<std::vector<Pair>> adm, inad;
  int l0 = 0;
};

void build_tree(const double* pts, int64_t N, int leafsize, Tree& t);
void build_partition(const Tree& t, double eta, Partition& p);
std::vector<std::vector<int>> near_lists(const Partition& p, int l);
std::vector<int> greedy_colours(const std::vector<std::vector<int>>& nbrs);

// H^2 representation in FP64, tree order, levels l0..L.
struct H2Host {
  Tree tree;
  Partition part;
  int L = 0, l0 = 0;
  std::vector<std::vector<int>> rank;                // [l][c]
  std::vector<std::vector<cplx>> V;                  // leaf bases, size x k
  std::vector<std::vector<std::vector<cplx>>> T;     // [l][c] (k1+k2) x k
  std::vector<std::vector<std::vector<cplx>>> S;     // [l][adm idx] kt x ks
  std::vector<std::vector<cplx>> D;                  // [inad[L] idx]
  std::vector<double> dscale;                        // global order (size N)
  bool symmetric = false;                            // Z^T = Z (h2_build; checked by h2_load)
  // construction phase times (h2_build), ms: far-field Grams, interpolative
  // decompositions + bases, couplings, dense near blocks
  double t_gram_ms = 0, t_id_ms = 0, t_coupling_ms = 0, t_near_ms = 0;
  // proxy construction: extra sample points after the N tree positions
  // (3 coordinates each) and their column weights (the sqrt(chi) slot)
  std::vector<double> proxy_pts, proxy_w;
};

// Far-field sample Grams of one level: G[t] = Z(rows[t], F) Z(rows[t], F)^H,
// rows in tree positions, F the tree-order ranges (start, count) of t.
using GramFn = std::function<void(int level, const std::vector<std::vector<int64_t>>& rows,
                                  const std::vector<std::vector<int64_t>>& ranges,
                                  std::vector<std::vector<cplx>>& G)>;

// H^2 construction (exact far-field sample + interpolative decomposition),
// h2_build.  `gram` computes the sample Grams (GPU kernel, or the host loop
// of host_only contexts).
std::string build_h2(const double* pts, int64_t N, double k, double h, const double* chi, int64_t chi_len,
                     double eps, const h2_opts& o, H2Host& H, const GramFn& gram);
std::vector<cplx> host_complement(const std::vector<cplx>& B, int n, int k);
// Z <- I + E (Z - I) E with E = diag(e), e in tree order (h2_set_chi)
void rescale_h2(H2Host& H, const std::vector<double>& e);
void host_gram(const double* pts_tree, const double* sq_tree, double k, double w,
               const std::vector<std::vector<int64_t>>& rows, const std::vector<std::vector<int64_t>>& ranges,
               std::vector<std::vector<cplx>>& G);

// ------------------------------------------------------------------------
// Device memory: grow-only buffers owned by the context.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void release();
};

struct Ctx;

// Error carried out of the host planners as an exception inside the library
// (converted to an h2_status at the ABI boundary).
struct Err {
  h2_status st;
  std::string msg;
};
[[noreturn]] void fail(h2_status st, const std::string& msg);
void ck(cudaError_t e, const char* what);

// Grow-only device buffer allocation with arena accounting.
void* dev_ensure(Ctx& c, DevBuf& b, size_t bytes);
// Frees a buffer of the context's arena accounting.
void dev_free(Ctx& c, DevBuf& b);
// allocation registry and the host-side bounds checks of the task lists
// (checks.cpp; on when H2_CHECKS is set in the environment)
bool checks_on();
void alloc_register(const void* p, size_t bytes);
void alloc_unregister(const void* p);
void check_range(const void* p, size_t bytes, const std::string& what);
// Frees the factors of the last factorization and the factorization scratch
// (after a failed factorization: the context keeps its H^2 matrix only).
void drop_factors(Ctx& c);

// Task staging: host task arrays are appended into one growing byte buffer,
// copied into pinned memory and uploaded with cudaMemcpyAsync just before the
// launch that reads them.  Uploaded ranges are never overwritten until
// begin(), which the caller issues only while the stream is idle.
struct Stager {
  std::vector<unsigned char> host;
  size_t uploaded = 0;
  void* pinned = nullptr;
  size_t cap = 0;
  DevBuf dev;
  std::vector<size_t> offs;
  ~Stager();
  void begin() { host.clear(); offs.clear(); uploaded = 0; }
  void swap(Stager& o) {
    host.swap(o.host);
    std::swap(uploaded, o.uploaded);
    std::swap(pinned, o.pinned);
    std::swap(cap, o.cap);
    DevBuf t = std::move(dev);
    dev = std::move(o.dev);
    o.dev = std::move(t);
    offs.swap(o.offs);
  }
  template <class T>
  int add(const std::vector<T>& v) {
    size_t o = (host.size() + 255) & ~(size_t)255;
    host.resize(o + v.size() * sizeof(T) + 1);
    if (!v.empty()) std::memcpy(host.data() + o, v.data(), v.size() * sizeof(T));
    offs.push_back(o);
    return (int)offs.size() - 1;
  }
  void upload(Ctx& c);
  template <class T>
  const T* ptr(int i) const { return (const T*)((const unsigned char*)dev.p + offs[i]); }
};

// Factor data of one level.
struct LevelF {
  int l = 0, nc = 0;
  // block LDL^T form (h2_opts.ldlt): pairs (a, b) with a > b are not stored;
  // their offsets point at the stored (b, a), read transposed
  bool sym = false;
  size_t near_elems = 0, fill_elems = 0;      // stored entries
  std::vector<int> n, k0, kt, m;
  std::vector<std::vector<int>> nbrs;          // near lists incl. self
  std::vector<std::vector<int>> batches;       // elimination batches
  std::vector<int> batch_of;
  std::vector<Pair> near_pairs;                // == part.inad[l]
  std::unordered_map<int64_t, int> near_id;
  std::vector<size_t> near_off;                // element offsets
  std::vector<Pair> fill_pairs;
  std::unordered_map<int64_t, int> fill_id;
  std::vector<size_t> fill_off;
  std::vector<char> fill_live;
  std::vector<std::vector<int>> fill_row, fill_col;  // fill pairs by row / column cluster
  std::vector<char> fill_is_adm;
  std::vector<size_t> B_off, Q_off, inv_off, piv_off, Vp_off;
  std::vector<double> snorm2;
  // near field, Q~, L^{-1}P and U^{-1}, pivots, eq. 35 panels: kept for the
  // solves; the fill-ins and the FP64 incoming bases / complements are only
  // needed while the level (and its merge) runs and live in the context's
  // ping-pong arenas (slot = level parity), shared by all levels
  DevBuf near_buf, Q_buf, inv_buf, piv_buf, Ub_buf;
  char* fill_ptr = nullptr;
  h2k::cd* B_ptr = nullptr;
  h2k::cd* Vp_ptr = nullptr;
  std::vector<size_t> Ub_off;                  // per (cluster, nbr) for eq. 35
  std::vector<int> nbr_first;                  // first (cluster, nbr) index
  // Step-0 statistics: Ritz subspace sizes and Jacobi sweeps
  int st_ritz_max = 0, st_ritz_n = 0, st_sweeps_max = 0;
  long st_ritz_sum = 0;
  // solve-time vector layout
  std::vector<int64_t> voff;                   // cluster offsets in level vector
  int64_t vlen = 0;
};

// Blocked LU of the final block (Algorithm 1, last line).
struct RootF {
  int n = 0, nb = 32;
  DevBuf R, piv, Linv, Uinv, Rinv;  // R packed LU; per-panel inverses
  std::vector<int> kt;               // kept sizes of the level-l0 clusters
};

struct Stats {
  int stop_level = -1;  // last factorized level of the last factorization
  double t_factor_ms = 0, t_solve_ms = 0, t_build_ms = 0;
  double t_sync_ms = 0;  // factorization: host time blocked in stream synchronizes
  double flops_factor = 0;
  int64_t launches_factor = 0, launches_solve = 0;
  int refine_iters = 0;
  double refine_resid = 0;
  std::vector<std::string> level_json;
};

// Optional per-launch timing (h2_opts.profile): CUDA events on the launch
// stream around each kernel, resolved after the call's final synchronize.
struct ProfRec {
  std::string tag;
  cudaEvent_t a, b;
  double flops;
  const char* pipe;  // arithmetic unit of the products, else null
  double bytes;      // algorithmic bytes (memory-bound classes), else 0
};
struct ProfAgg {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
  const char* pipe = nullptr;
};

// A second stream of the context for work that overlaps the main stream's
// (the fill-in trace of Step 0), with the two events that order it.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  SideStream() = default;
  SideStream(const SideStream&) = delete;
  SideStream& operator=(const SideStream&) = delete;
  ~SideStream() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
  }
};

struct Ctx {
  H2Host H;
  cudaStream_t stream = nullptr;
  SideStream side;
  // the FP64 matvec's products in double-float while set (MvEmul)
  bool mv_emul = false;
  h2_opts opts;
  std::string err;
  size_t dev_bytes = 0, dev_peak = 0;
  // device copy of the H^2 (FP64)
  DevBuf dV, dT, dS, dD, dperm, dscale, dVp, dTp;
  std::vector<size_t> V_off, Vp_off;                // per leaf
  std::vector<std::vector<size_t>> Tp_off;          // complements of T
  std::vector<std::vector<size_t>> T_off, S_off;    // [l][c] / [l][adm idx]
  std::vector<size_t> D_off;                        // per inad[L] pair
  std::vector<std::unordered_map<int64_t, int>> adm_id;  // [l] pair -> idx
  // factorization
  bool factored = false, inverted = false;
  bool fac_ldlt = false;  // the factors are in block LDL^T form (h2_opts.ldlt)
  int prec = 0;
  double eps_fill = 0;
  // CUDA-graph replay of solves: a graph is valid while no device buffer of
  // its instances was (re)allocated (gen) and none was refactorized (epoch)
  uint64_t gen = 0, epoch = 0;
  bool capturing = false;
  std::vector<std::unique_ptr<struct SolveGraph>> graphs;
  std::vector<LevelF> lev;  // lev[0] = leaf level L, ..., last = l0
  RootF root;
  // scratch
  DevBuf scratch, scratch2, vecbuf, vecbuf2, vecbuf3, normbuf, statusbuf, gemm_ws, jac_buf, applybuf, frobbuf;
  DevBuf fill_pp[2], B_pp[2], Vp_pp[2];  // per-level working arenas, by level parity
  DevBuf lu_scr;                         // partial-LU inversion scratch of one batch
  DevBuf ldlt_w;                         // block LDL^T: F^-1 Z_i'k of one batch
  Stager st;
  Stats stats;
  int64_t launches = 0;
  std::vector<ProfRec> prof_open;
  std::vector<cudaEvent_t> prof_pool;
  std::unordered_map<std::string, ProfAgg> prof;  // per kernel class, since the last reset
  // launches per code path variant (kernel, arithmetic unit, tile shape, CTAs
  // per thread-block cluster), counted since the context was created
  std::map<std::string, int64_t> paths;
  std::string prof_suffix;                        // profile == 2: "@<level>" appended to tags
  // sum of ||S||_F^2 over the admissible blocks of each cluster's row and
  // column, per level (depends on the H^2 only; computed once)
  std::vector<std::vector<double>> snorm2_cache;
  std::vector<std::vector<int>> colour_cache;  // near-field colouring per level
  // early stop at level cov_level > l0: couplings of the level's pairs that
  // lie inside an ancestor's admissible block, E_a S E_b^T (FP64, k_a x k_b)
  int cov_level = -1;
  DevBuf cov_buf, cov_E, cov_Y;
  std::unordered_map<int64_t, size_t> cov_off;
};

// A captured forward / backward (or adjoint) sweep of a group of instances:
// its task lists live in its own staging buffers, so replays need no host
// planning.  Owned by the group's first context.
struct SolveGraph {
  std::vector<Ctx*> cs;
  std::vector<void*> xs;
  int nrhs = 0;
  bool adjoint = false, inverse = false;
  std::vector<uint64_t> gens, epochs;
  Stager st;
  cudaGraphExec_t exec = nullptr;
  int64_t nlaunch = 0;  // kernels per replay
  ~SolveGraph();
};

// Host wall time of a planning phase, kept as class "host:<tag>" (profile == 2)
struct HostScope {
  Ctx& c;
  const char* tag;
  std::chrono::steady_clock::time_point t0;
  HostScope(Ctx& c_, const char* tag_) : c(c_), tag(tag_), t0(std::chrono::steady_clock::now()) {}
  ~HostScope();
};

// RAII bracket of one kernel launch (no-op unless opts.profile)
struct ProfScope {
  Ctx& c;
  bool on;
  size_t idx = 0;
  ProfScope(Ctx& c_, const std::string& tag, double flops, const char* pipe = nullptr, double bytes = 0.0);
  ~ProfScope();
};
// Scope in which the FP64 H^2 matvec stages of `c` run their products in
// double-float on the FP32 pipe (h2_opts.matvec_emulation).
struct MvEmul {
  Ctx& c;
  bool old;
  MvEmul(Ctx& cc, bool on) : c(cc), old(cc.mv_emul) { c.mv_emul = on; }
  ~MvEmul() { c.mv_emul = old; }
  MvEmul(const MvEmul&) = delete;
  MvEmul& operator=(const MvEmul&) = delete;
};

void prof_resolve(Ctx& c);  // after a stream synchronize: fold events into c.prof
// cudaStreamSynchronize with the blocked host time added to c.stats.t_sync_ms
void sync_timed(Ctx& c, cudaStream_t s, const char* what);
void prof_reset(Ctx& c);

// accessors of the ABI context object (defined with it in api.cpp)
Ctx* ctx_core(h2_ctx* x);
const double* ctx_invscale(h2_ctx* x);

void upload_h2(Ctx& c);
void factorize(Ctx& c, double eps, int prec);
// Several independent instances in lockstep (launches on cs[0]'s stream)
void factorize_group(const std::vector<Ctx*>& cs, double eps, int prec);
void solve_tree_group(const std::vector<Ctx*>& cs, const std::vector<void*>& xs, int nrhs, bool adjoint,
                      bool use_inverse);
// blocked-LU solve with the final blocks of several instances (same nrhs)
void root_solve_grouped(Ctx& lc, const std::vector<Ctx*>& cs, const std::vector<char*>& xs,
                        const std::vector<int>& lds, int nrhs, bool adjoint);
void matvec_tree_group(const std::vector<Ctx*>& cs, const std::vector<const h2k::cd*>& xs,
                       const std::vector<h2k::cd*>& ys, int nrhs, bool adjoint);
void invert(Ctx& c);
// x (tree order, bulk precision vector of length N*nrhs) <- Z^{-1} x in place
void solve_tree(Ctx& c, void* x, int nrhs, bool adjoint, bool use_inverse);
// y = Z_H2 x, FP64, tree order
void matvec_tree(Ctx& c, const h2k::cd* x, h2k::cd* y, int nrhs, bool adjoint);

}  // namespace h2
