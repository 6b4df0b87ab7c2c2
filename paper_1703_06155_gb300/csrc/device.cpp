// Device memory, task staging, and the FP64 device copy of the H^2 matrix.
#include <cstdlib>
#include <cuda_runtime.h>

#include <algorithm>

#include <chrono>

#include "h2_host.h"

namespace h2 {

void DevBuf::release() {
  if (p) {
    alloc_unregister(p);
    cudaFree(p);
  }
  p = nullptr;
  bytes = 0;
}

[[noreturn]] void fail(h2_status st, const std::string& msg) { throw Err{st, msg}; }

static cudaEvent_t prof_event(Ctx& c) {
  if (!c.prof_pool.empty()) {
    cudaEvent_t e = c.prof_pool.back();
    c.prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  ck(cudaEventCreate(&e), "cudaEventCreate");
  return e;
}

ProfScope::ProfScope(Ctx& c_, const std::string& tag, double flops, const char* pipe, double bytes)
    : c(c_), on(c_.opts.profile != 0 && !c_.capturing) {
  if (!on) return;
  ProfRec r{c.opts.profile == 2 ? tag + c.prof_suffix : tag, prof_event(c), prof_event(c), flops, pipe, bytes};
  ck(cudaEventRecord(r.a, c.stream), "cudaEventRecord");
  idx = c.prof_open.size();
  c.prof_open.push_back(r);
}

ProfScope::~ProfScope() {
  if (on) cudaEventRecord(c.prof_open[idx].b, c.stream);
}

void prof_resolve(Ctx& c) {
  for (ProfRec& r : c.prof_open) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ProfAgg& a = c.prof[r.tag];
      a.launches++;
      a.ms += ms;
      a.flops += r.flops;
      a.bytes += r.bytes;
      if (r.pipe) a.pipe = r.pipe;
    } else {
      cudaGetLastError();
    }
    c.prof_pool.push_back(r.a);
    c.prof_pool.push_back(r.b);
  }
  c.prof_open.clear();
}

void prof_reset(Ctx& c) { c.prof.clear(); }

HostScope::~HostScope() {
  if (c.opts.profile != 2) return;
  ProfAgg& a = c.prof[std::string("host:") + tag + c.prof_suffix];
  a.launches++;
  a.ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(H2_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void sync_timed(Ctx& c, cudaStream_t s, const char* what) {
  const auto t0 = std::chrono::steady_clock::now();
  ck(cudaStreamSynchronize(s), what);
  c.stats.t_sync_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void* dev_ensure(Ctx& c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (b.bytes >= bytes) return b.p;
  const size_t old = b.bytes;
  const size_t want = std::max(bytes, old + old / 4);
  if (c.capturing) fail(H2_EINTERNAL, "device allocation during graph capture");
  if (c.opts.arena_cap_bytes && c.dev_bytes - old + want > c.opts.arena_cap_bytes)
    fail(H2_ENOMEM, "device arena cap exceeded");
  // the old contents are not kept: grow-only scratch / per-factorization arenas
  if (b.p) {
    ck(cudaStreamSynchronize(c.stream), "sync before realloc");
    if (c.side.s) ck(cudaStreamSynchronize(c.side.s), "sync before realloc");
    alloc_unregister(b.p);
    cudaFree(b.p);
    b.p = nullptr;
    c.dev_bytes -= old;
    b.bytes = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    fail(H2_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
  }
  // debugging aid: H2_POISON_ALLOC set in the environment fills every new
  // buffer with 0xFF bytes (NaN in every floating-point type), so that a
  // kernel reading memory nothing has written yet shows up as NaN results
  static const bool poison = std::getenv("H2_POISON_ALLOC") != nullptr;
  if (poison) ck(cudaMemsetAsync(p, 0xFF, want, c.stream), "poison");
  alloc_register(p, want);
  b.p = p;
  b.bytes = want;
  c.gen++;
  c.dev_bytes += want;
  c.dev_peak = std::max(c.dev_peak, c.dev_bytes);
  return p;
}

void dev_free(Ctx& c, DevBuf& b) {
  if (!b.p) return;
  c.dev_bytes -= b.bytes;
  b.release();
  c.gen++;
}

void drop_factors(Ctx& c) {
  cudaStreamSynchronize(c.stream);  // nothing of the failed call may still use the buffers
  cudaGetLastError();
  for (LevelF& F : c.lev)
    for (DevBuf* b : {&F.near_buf, &F.Q_buf, &F.inv_buf, &F.piv_buf, &F.Ub_buf}) dev_free(c, *b);
  c.lev.clear();
  for (DevBuf* b : {&c.root.R, &c.root.piv, &c.root.Linv, &c.root.Uinv, &c.root.Rinv}) dev_free(c, *b);
  c.root = RootF();
  for (DevBuf* b : {&c.scratch, &c.scratch2, &c.gemm_ws, &c.jac_buf, &c.applybuf, &c.frobbuf, &c.lu_scr,
                    &c.fill_pp[0], &c.fill_pp[1], &c.B_pp[0], &c.B_pp[1], &c.Vp_pp[0], &c.Vp_pp[1]})
    dev_free(c, *b);
  c.factored = false;
  c.inverted = false;
  c.graphs.clear();
}

Stager::~Stager() {
  if (pinned) cudaFreeHost(pinned);
}

SolveGraph::~SolveGraph() {
  if (exec) cudaGraphExecDestroy(exec);
}

void Stager::upload(Ctx& c) {
  if (uploaded >= host.size()) return;
  if (cap < host.size()) {
    // everything uploaded so far has been consumed by launches already in
    // the stream: wait for them, grow, and upload the whole range again
    ck(cudaStreamSynchronize(c.stream), "stager sync");
    if (c.side.s) ck(cudaStreamSynchronize(c.side.s), "stager sync");
    if (pinned) cudaFreeHost(pinned);
    pinned = nullptr;
    cap = std::max(host.size() * 2, (size_t)1 << 20);
    ck(cudaMallocHost(&pinned, cap), "cudaMallocHost");
    dev_ensure(c, dev, cap);
    uploaded = 0;
  }
  std::memcpy((unsigned char*)pinned + uploaded, host.data() + uploaded, host.size() - uploaded);
  ck(cudaMemcpyAsync((unsigned char*)dev.p + uploaded, (unsigned char*)pinned + uploaded, host.size() - uploaded,
                     cudaMemcpyHostToDevice, c.stream),
     "task upload");
  uploaded = host.size();
}

template <class T>
static void upload_vec(Ctx& c, DevBuf& b, const std::vector<T>& v) {
  dev_ensure(c, b, v.size() * sizeof(T));
  if (!v.empty()) ck(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c.stream), "upload");
  ck(cudaStreamSynchronize(c.stream), "upload sync");
}

void upload_h2(Ctx& c) {
  H2Host& H = c.H;
  const int L = H.L, l0 = H.l0;
  std::vector<cplx> buf;
  // leaf bases
  c.V_off.assign(size_t(1) << L, 0);
  for (int t = 0; t < (1 << L); ++t) {
    c.V_off[t] = buf.size();
    buf.insert(buf.end(), H.V[t].begin(), H.V[t].end());
  }
  upload_vec(c, c.dV, buf);
  buf.clear();
  c.T_off.assign(L + 1, {});
  for (int l = l0; l < L; ++l) {
    c.T_off[l].assign(size_t(1) << l, 0);
    for (int t = 0; t < (1 << l); ++t) {
      c.T_off[l][t] = buf.size();
      buf.insert(buf.end(), H.T[l][t].begin(), H.T[l][t].end());
    }
  }
  upload_vec(c, c.dT, buf);
  buf.clear();
  c.S_off.assign(L + 1, {});
  c.adm_id.assign(L + 1, {});
  for (int l = l0; l <= L; ++l) {
    c.S_off[l].assign(H.part.adm[l].size(), 0);
    for (size_t q = 0; q < H.part.adm[l].size(); ++q) {
      c.S_off[l][q] = buf.size();
      buf.insert(buf.end(), H.S[l][q].begin(), H.S[l][q].end());
      c.adm_id[l][pkey(H.part.adm[l][q].first, H.part.adm[l][q].second)] = (int)q;
    }
  }
  upload_vec(c, c.dS, buf);
  buf.clear();
  c.D_off.assign(H.part.inad[L].size(), 0);
  for (size_t q = 0; q < H.part.inad[L].size(); ++q) {
    c.D_off[q] = buf.size();
    buf.insert(buf.end(), H.D[q].begin(), H.D[q].end());
  }
  upload_vec(c, c.dD, buf);
  // complements of the leaf bases and of the transfer matrices (Step 1)
  buf.clear();
  c.Vp_off.assign(size_t(1) << L, 0);
  for (int t = 0; t < (1 << L); ++t) {
    c.Vp_off[t] = buf.size();
    const int n = (int)H.tree.size[L][t], k = H.rank[L][t];
    const std::vector<cplx> E = host_complement(H.V[t], n, k);
    buf.insert(buf.end(), E.begin(), E.end());
  }
  upload_vec(c, c.dVp, buf);
  buf.clear();
  c.Tp_off.assign(L + 1, {});
  for (int l = l0; l < L; ++l) {
    c.Tp_off[l].assign(size_t(1) << l, 0);
    for (int t = 0; t < (1 << l); ++t) {
      c.Tp_off[l][t] = buf.size();
      const int n = H.rank[l + 1][2 * t] + H.rank[l + 1][2 * t + 1], k = H.rank[l][t];
      const std::vector<cplx> E = host_complement(H.T[l][t], n, k);
      buf.insert(buf.end(), E.begin(), E.end());
    }
  }
  upload_vec(c, c.dTp, buf);
  upload_vec(c, c.dperm, H.tree.perm);
  upload_vec(c, c.dscale, H.dscale);
}

}  // namespace h2
