// Host-side bounds checks of the planned task lists.
//
// With H2_CHECKS set in the environment every batched launch (GEMM, copy,
// apply and partial-LU task lists) first checks, on the host, that each
// device range a task reads or writes lies inside a single allocation the
// library made; a range that overruns its allocation, or starts in none,
// fails the call with H2_EINTERNAL and a message naming the launch and the
// task.  This catches planning mistakes (a wrong offset or leading
// dimension) before a kernel can touch memory it does not own, on the host
// and without any device-side cost.  The registry of allocations is kept
// whether or not the checks are on (a map insert per allocation).
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "batch.h"
#include "h2_host.h"

namespace h2 {
namespace {

std::mutex g_mu;
std::map<uintptr_t, size_t>& allocs() {
  static std::map<uintptr_t, size_t> m;
  return m;
}

size_t es_of(int prec) { return prec == h2k::P64 ? sizeof(h2k::cd) : sizeof(h2k::cf); }

// bytes spanned by a column-major rows x cols block with leading dimension ld
size_t span(int64_t rows, int64_t cols, int64_t ld, size_t es) {
  if (rows <= 0 || cols <= 0) return 0;
  return (size_t)((cols - 1) * ld + rows) * es;
}

}  // namespace

bool checks_on() {
  static const bool on = std::getenv("H2_CHECKS") != nullptr;
  return on;
}

void alloc_register(const void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_mu);
  allocs()[(uintptr_t)p] = bytes;
}

void alloc_unregister(const void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_mu);
  allocs().erase((uintptr_t)p);
}

void check_range(const void* p, size_t bytes, const std::string& what) {
  if (!p || bytes == 0) return;
  const uintptr_t a = (uintptr_t)p;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = allocs().upper_bound(a);
  if (it == allocs().begin()) fail(H2_EINTERNAL, "bounds check: " + what + " starts outside every allocation");
  --it;
  const uintptr_t base = it->first, end = base + it->second;
  if (a >= end) fail(H2_EINTERNAL, "bounds check: " + what + " starts outside every allocation");
  if (a + bytes > end)
    fail(H2_EINTERNAL, "bounds check: " + what + " overruns its allocation by " + std::to_string(a + bytes - end) +
                           " bytes");
}

void check_gemm(const GemmBatch& b, int pina, int pin, int pout, const char* what) {
  const size_t ea = es_of(pina < 0 ? pin : pina), eb = es_of(pin), ec = es_of(pout);
  for (size_t ti = 0; ti < b.t.size(); ++ti) {
    const h2k::GemmTask& g = b.t[ti];
    const std::string tag = std::string(what) + " task " + std::to_string(ti);
    check_range(g.C, span(g.M, g.N, g.ldc, ec), tag + " C");
    for (int q = g.p0; q < g.p0 + g.np; ++q) {
      const h2k::GemmPair& pr = b.p[q];
      const bool at = pr.opA == h2k::OP_T || pr.opA == h2k::OP_H, bt = pr.opB == h2k::OP_T || pr.opB == h2k::OP_H;
      check_range(pr.A, at ? span(pr.K, g.M, pr.lda, ea) : span(g.M, pr.K, pr.lda, ea), tag + " A");
      check_range(pr.B, bt ? span(g.N, pr.K, pr.ldb, eb) : span(pr.K, g.N, pr.ldb, eb), tag + " B");
    }
  }
}

void check_copy(const CopyBatch& b, const char* what) {
  for (size_t i = 0; i < b.t.size(); ++i) {
    const h2k::CopyTask& t = b.t[i];
    const std::string tag = std::string(what) + " copy " + std::to_string(i);
    if (t.mode != 2 && t.src) {
      const int r = std::min(t.rows, t.srows), c = std::min(t.cols, t.scols);
      check_range(t.src, t.transpose ? span(c, r, t.lds, es_of(t.src_prec)) : span(r, c, t.lds, es_of(t.src_prec)),
                  tag + " source");
    }
    check_range(t.dst, span(t.rows, t.cols, t.ldd, es_of(t.dst_prec)), tag + " destination");
  }
}

void check_apply(const ApplyBatch& b, bool left, int prec, const char* what) {
  const size_t es = es_of(prec);
  for (size_t i = 0; i < b.t.size(); ++i) {
    const h2k::ApplyTask& t = b.t[i];
    const std::string tag = std::string(what) + " apply " + std::to_string(i);
    check_range(t.A, span(t.p, t.p, t.lda, es), tag + " A");
    check_range(t.X, left ? span(t.p, t.w, t.ldx, es) : span(t.w, t.p, t.ldx, es), tag + " X");
  }
}

void check_lu(const std::vector<h2k::LuTask>& lu, int prec) {
  const size_t es = es_of(prec);
  for (size_t i = 0; i < lu.size(); ++i) {
    const h2k::LuTask& t = lu[i];
    const std::string tag = "partial LU " + std::to_string(i);
    check_range(t.A, span(t.m, t.m, t.lda, es), tag + " A");
    check_range(t.Linv, span(t.m, t.m, t.m, es), tag + " L^-1 P");
    check_range(t.Uinv, span(t.m, t.m, t.m, es), tag + " U^-1");
    check_range(t.scratch, span(t.m, t.m, t.m, es), tag + " scratch");
    check_range(t.piv, (size_t)t.m * sizeof(int), tag + " pivots");
  }
}

}  // namespace h2
