// h2_matvec_noalloc: the FP64 H^2 matrix-vector product of h2_matvec, for
// callers that must not allocate device memory during the call (for example a
// real-time loop or a host thread that owns no allocator: the context was set
// up earlier, the per-call work may not cudaMalloc).  All temporaries of the
// product -- the permuted and scaled input and output vectors, the level
// coefficient vectors of the upward / downward passes, and the task
// descriptors of the batched GEMM launches -- live in one file-scope device
// array of fixed size, shared by every call in the process.
//
// The array's host-side name is only a stand-in: its device address is taken
// once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernels.  With CUDA's lazy module loading (the default since
// CUDA 12.2) that lookup is also what loads this file's module on the device,
// so the 32 MiB are reserved at the first call on each device, not when the
// library is loaded.
#include <mutex>
#include <unordered_map>

#include "batch.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;  // 32 MiB per device

__device__ __align__(256) unsigned char g_h2_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
std::unordered_map<int, void*> g_addr;  // device ordinal -> device address

// First call on a device: resolve the array's device address (no allocation).
void* scratch_address(std::string& err) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    err = "cudaGetDevice failed";
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_addr.find(dev);
  if (it != g_addr.end()) return it->second;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_h2_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    err = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
    return nullptr;
  }
  g_addr[dev] = p;
  return p;
}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

using namespace h2;
using namespace h2k;

static h2_status matvec_noalloc(h2_ctx* ctx, const void* xin, void* yout, int nrhs, unsigned flags, void* stream) {
  if (!ctx) return H2_EINVAL;
  Ctx& c = *ctx_core(ctx);
  if (c.opts.host_only) {
    c.err = "context was built with host_only";
    return H2_ESTATE;
  }
  if (!xin || !yout || nrhs <= 0 || xin == yout || (flags & ~H2_ADJOINT)) {
    c.err = "h2_matvec_noalloc: bad argument (device x, y distinct; nrhs > 0; flags: H2_ADJOINT only)";
    return H2_EINVAL;
  }
  for (const void* v : {xin, (const void*)yout}) {
    cudaPointerAttributes at{};
    const cudaError_t pe = cudaPointerGetAttributes(&at, v);
    if (pe != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      c.err = "h2_matvec_noalloc: x and y must be device (or managed) memory";
      return H2_EINVAL;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      c.err = "h2_matvec_noalloc: cudaStreamIsCapturing failed";
      return H2_ECUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) {
      c.err = "h2_matvec_noalloc: the stream is being captured (the call uploads its task lists from host memory "
              "and synchronizes the stream); nothing was enqueued";
      return H2_ESTATE;
    }
  }
  const bool adj = flags & H2_ADJOINT;
  const H2Host& H = c.H;
  const int L = H.L, l0 = H.l0;
  const int64_t N = H.tree.N;
  std::string err;
  unsigned char* base = (unsigned char*)scratch_address(err);
  if (!base) {
    c.err = "h2_matvec_noalloc: " + err;
    return H2_ECUDA;
  }
  // ---- layout of the static array -------------------------------------
  std::vector<std::vector<size_t>> koff(L + 1);
  std::vector<size_t> K(L + 1, 0), lb(L + 1, 0);
  size_t ktot = 0;
  for (int l = l0; l <= L; ++l) {
    koff[l].assign(size_t(1) << l, 0);
    for (int t = 0; t < (1 << l); ++t) {
      koff[l][t] = K[l];
      K[l] += H.rank[l][t];
    }
    lb[l] = ktot;
    ktot += K[l] * nrhs;
  }
  const size_t vbytes = align256((size_t)N * nrhs * sizeof(cd));
  const size_t hbytes = align256(ktot * sizeof(cd));
  size_t off = 0;
  cd* t1 = (cd*)(base + off);
  off += vbytes;
  cd* t2 = (cd*)(base + off);
  off += vbytes;
  cd* xhb = (cd*)(base + off);
  off += hbytes;
  cd* yhb = (cd*)(base + off);
  off += hbytes;
  const size_t task_base = off;
  auto xh = [&](int l, int t) { return xhb + lb[l] + koff[l][t]; };
  auto yh = [&](int l, int t) { return yhb + lb[l] + koff[l][t]; };
  const cd* Vd = (const cd*)c.dV.p;
  const cd* Td = (const cd*)c.dT.p;
  const cd* Sd = (const cd*)c.dS.p;
  const cd* Dd = (const cd*)c.dD.p;
  const int opUp = adj ? OP_H : OP_T, opDown = adj ? OP_C : OP_N;
  // ---- the same stages as h2_matvec, one GEMM batch each ---------------
  std::vector<GemmBatch> stages;
  {
    GemmBatch g;
    for (int t = 0; t < (1 << L); ++t) {
      const int kt = H.rank[L][t], nt = (int)H.tree.size[L][t];
      if (kt == 0) continue;
      g.task(xh(L, t), (int)K[L], kt, nrhs, 1.0, 0.0);
      g.pair(Vd + c.V_off[t], nt, opUp, t1 + H.tree.start[L][t], (int)N, OP_N, nt);
      g.close();
    }
    stages.push_back(std::move(g));
  }
  for (int l = L - 1; l >= l0; --l) {
    GemmBatch g;
    for (int t = 0; t < (1 << l); ++t) {
      const int kt = H.rank[l][t], k1 = H.rank[l + 1][2 * t], k2 = H.rank[l + 1][2 * t + 1];
      if (kt == 0) continue;
      g.task(xh(l, t), (int)K[l], kt, nrhs, 1.0, 0.0);
      g.pair(Td + c.T_off[l][t], k1 + k2, opUp, xh(l + 1, 2 * t), (int)K[l + 1], OP_N, k1 + k2);
      g.close();
    }
    stages.push_back(std::move(g));
  }
  {
    GemmBatch g;
    for (int l = l0; l <= L; ++l) {
      std::vector<std::vector<int>> by(size_t(1) << l);
      for (size_t q = 0; q < H.part.adm[l].size(); ++q) by[adj ? H.part.adm[l][q].second : H.part.adm[l][q].first].push_back((int)q);
      for (int u = 0; u < (1 << l); ++u) {
        const int ku = H.rank[l][u];
        if (ku == 0) continue;
        g.task(yh(l, u), (int)K[l], ku, nrhs, 1.0, 0.0);
        for (int q : by[u]) {
          const auto [t, s2] = H.part.adm[l][q];
          if (!adj) g.pair(Sd + c.S_off[l][q], H.rank[l][t], OP_N, xh(l, s2), (int)K[l], OP_N, H.rank[l][s2]);
          else g.pair(Sd + c.S_off[l][q], H.rank[l][t], OP_H, xh(l, t), (int)K[l], OP_N, H.rank[l][t]);
        }
        g.close();
      }
    }
    stages.push_back(std::move(g));
  }
  for (int l = l0; l < L; ++l) {
    GemmBatch g;
    for (int t = 0; t < (1 << l); ++t) {
      const int kt = H.rank[l][t], k1 = H.rank[l + 1][2 * t], k2 = H.rank[l + 1][2 * t + 1];
      if (kt == 0 || k1 + k2 == 0) continue;
      g.task(yh(l + 1, 2 * t), (int)K[l + 1], k1 + k2, nrhs, 1.0, 1.0);
      g.pair(Td + c.T_off[l][t], k1 + k2, opDown, yh(l, t), (int)K[l], OP_N, kt);
      g.close();
    }
    stages.push_back(std::move(g));
  }
  {
    std::vector<std::vector<int>> by(size_t(1) << L);
    for (size_t q = 0; q < H.part.inad[L].size(); ++q) by[adj ? H.part.inad[L][q].second : H.part.inad[L][q].first].push_back((int)q);
    GemmBatch g;
    for (int u = 0; u < (1 << L); ++u) {
      const int nu = (int)H.tree.size[L][u], ku = H.rank[L][u];
      g.task(t2 + H.tree.start[L][u], (int)N, nu, nrhs, 1.0, 0.0);
      if (ku > 0) g.pair(Vd + c.V_off[u], nu, opDown, yh(L, u), (int)K[L], OP_N, ku);
      for (int q : by[u]) {
        const auto [t, s2] = H.part.inad[L][q];
        const int nt = (int)H.tree.size[L][t], ns = (int)H.tree.size[L][s2];
        if (!adj) g.pair(Dd + c.D_off[q], nt, OP_N, t1 + H.tree.start[L][s2], (int)N, OP_N, ns);
        else g.pair(Dd + c.D_off[q], nt, OP_H, t1 + H.tree.start[L][t], (int)N, OP_N, nt);
      }
      g.close();
    }
    stages.push_back(std::move(g));
  }
  // ---- task descriptors into the static array (no split-K workspace) -----
  std::vector<unsigned char> host;
  struct Off { size_t t, p, tl; };
  std::vector<Off> offs;
  for (GemmBatch& g : stages) {
    g.plan(0);  // one K chunk per tile: no workspace
    Off o{};
    auto put = [&](const void* src, size_t bytes) {
      const size_t at = align256(host.size());
      host.resize(at + bytes);
      if (bytes) std::memcpy(host.data() + at, src, bytes);
      return at;
    };
    o.t = put(g.t.data(), g.t.size() * sizeof(GemmTask));
    o.p = put(g.p.data(), g.p.size() * sizeof(GemmPair));
    o.tl = put(g.tl.data(), g.tl.size() * sizeof(GemmTile));
    offs.push_back(o);
  }
  // one bound on the whole layout (vectors, level coefficients, task lists),
  // checked before anything is enqueued; the stage pointers computed above
  // are not dereferenced on the host
  if (task_base + host.size() > kNoAllocBytes) {
    c.err = "h2_matvec_noalloc: problem too large for the " + std::to_string(kNoAllocBytes >> 20) +
            " MiB static scratch (needs " + std::to_string((task_base + host.size() + (1 << 20) - 1) >> 20) +
            " MiB: " + std::to_string(task_base >> 20) + " MiB of vectors, " + std::to_string(host.size() >> 10) +
            " KiB of task lists)";
    return H2_EINVAL;
  }
  unsigned char* dtask = base + task_base;
  auto fail_cuda = [&](cudaError_t e, const char* what) {
    c.err = std::string("h2_matvec_noalloc: ") + what + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return H2_ECUDA;
  };
  cudaError_t e = cudaMemcpyAsync(dtask, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail_cuda(e, "task upload");
  const double* sc = (const double*)c.dscale.p;
  const double* isc = ctx_invscale(ctx);
  e = permute_scale(xin, t1, (const int64_t*)c.dperm.p, adj ? isc : sc, N, nrhs, P64, P64, 0, 0, s);
  if (e != cudaSuccess) return fail_cuda(e, "permute");
  for (size_t i = 0; i < stages.size(); ++i) {
    const GemmBatch& g = stages[i];
    if (g.tl.empty()) continue;
    e = gemm((const GemmTask*)(dtask + offs[i].t), (const GemmPair*)(dtask + offs[i].p),
             (const GemmTile*)(dtask + offs[i].tl), (int)g.tl.size(), P64, P64, P64, nullptr, s, g.shape);
    if (e != cudaSuccess) return fail_cuda(e, "gemm");
  }
  e = permute_scale(t2, yout, (const int64_t*)c.dperm.p, adj ? sc : isc, N, nrhs, P64, P64, 1, 0, s);
  if (e != cudaSuccess) return fail_cuda(e, "permute");
  // the host task buffer must outlive the (pageable) upload
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "sync");
  c.err.clear();
  return H2_OK;
}

// Exceptions of the host-side planning (allocation of the host task lists,
// message strings) become an h2_status here: nothing throws across the ABI.
extern "C" h2_status h2_matvec_noalloc(h2_ctx* ctx, const void* xin, void* yout, int nrhs, unsigned flags,
                                       void* stream) {
  try {
    return matvec_noalloc(ctx, xin, yout, nrhs, flags, stream);
  } catch (const Err& e) {
    if (ctx) ctx_core(ctx)->err = "h2_matvec_noalloc: " + e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx_core(ctx)->err = "h2_matvec_noalloc: host allocation of the task lists failed";
    return H2_ENOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx_core(ctx)->err = std::string("h2_matvec_noalloc: internal: ") + e.what();
    return H2_EINTERNAL;
  } catch (...) {
    if (ctx) ctx_core(ctx)->err = "h2_matvec_noalloc: internal error";
    return H2_EINTERNAL;
  }
}
