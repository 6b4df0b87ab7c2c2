// One-CTA-per-matrix dense kernels of the factorization and small vector
// helpers.
//
//  householder_complement  Step 1 (eqs. 4, 19, 28): orthonormal complement of
//                          an orthonormal cluster basis by Householder QR
//  jacobi_eig              Step 0 (eqs. 17, 26): eigen-decomposition of the
//                          fill-in Gram in complement coordinates (FP64)
//
// (The partial LU of Step 3 is in lu.cu.)
//
// Reductions use warp shuffles and a shared-memory stage.  The Jacobi sweep
// loop is bounded (kMaxSweeps); a matrix that does not converge within it
// reports status 2 to the host instead of spinning.
#include "h2_kernels.h"

namespace h2k {
namespace {

constexpr int NT = 256;
constexpr int kMaxSweeps = 60;

template <class E> struct RealOf;
template <> struct RealOf<cd> { using T = double; };
template <> struct RealOf<cf> { using T = float; };

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class R>
__device__ R block_sum(R v, R* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  R t = 0;
  if (threadIdx.x < 32) {
    t = (l < (int)(blockDim.x >> 5)) ? red[l] : (R)0;
    t = warp_sum(t);
    if (l == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// ----------------------------------------------------------------------------
// Householder complement (FP64). W <- B; for j < k: reflector H_j with
// H_j^H W[j:, j] = beta e_1 (LAPACK zlarfg convention, H = I - tau v v^H,
// v_0 = 1); apply H_j^H to the trailing columns. Then Vp = H_0 ... H_{k-1}
// [0; I_{n-k}].
__global__ void __launch_bounds__(NT) k_householder(const HhTask* __restrict__ tasks) {
  __shared__ double red[32];
  __shared__ double tau_r[1024], tau_i[1024];
  const HhTask t = tasks[blockIdx.x];
  const int n = t.n, k = t.k;
  cd* W = t.W;
  cd* Vp = t.Vp;
  for (int idx = threadIdx.x; idx < n * k; idx += NT) W[idx] = t.B[idx];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = NT / 32;
  for (int j = 0; j < k; ++j) {
    double s = 0;
    for (int i = j + 1 + threadIdx.x; i < n; i += NT) {
      const cd v = W[i + (size_t)j * n];
      s += v.re * v.re + v.im * v.im;
    }
    s = block_sum(s, red);
    const cd al = W[j + (size_t)j * n];
    double tr = 0, ti = 0, scr = 0, sci = 0;
    if (!(s == 0.0 && al.im == 0.0)) {
      const double nrm = sqrt(al.re * al.re + al.im * al.im + s);
      const double beta = al.re >= 0 ? -nrm : nrm;
      tr = (beta - al.re) / beta;
      ti = -al.im / beta;
      // scale = 1 / (alpha - beta)
      const double dr = al.re - beta, di = al.im;
      const double dd = dr * dr + di * di;
      scr = dr / dd;
      sci = -di / dd;
      for (int i = j + 1 + threadIdx.x; i < n; i += NT) {
        cd v = W[i + (size_t)j * n];
        const double vr = v.re * scr - v.im * sci, vi = v.re * sci + v.im * scr;
        v.re = vr;
        v.im = vi;
        W[i + (size_t)j * n] = v;
      }
    }
    if (threadIdx.x == 0) { tau_r[j] = tr; tau_i[j] = ti; }
    __syncthreads();
    if (tr == 0.0 && ti == 0.0) continue;
    // apply H^H = I - conj(tau) v v^H to columns j+1..k-1
    for (int c = j + 1 + warp; c < k; c += nw) {
      double dr = 0, di = 0;  // d = v^H W[:, c]
      for (int i = j + lane; i < n; i += 32) {
        const cd w = W[i + (size_t)c * n];
        cd v;
        if (i == j) { v.re = 1; v.im = 0; } else v = W[i + (size_t)j * n];
        dr += v.re * w.re + v.im * w.im;
        di += v.re * w.im - v.im * w.re;
      }
      dr = warp_sum(dr);
      di = warp_sum(di);
      // f = conj(tau) * d
      const double fr = tr * dr + ti * di, fi = tr * di - ti * dr;
      for (int i = j + lane; i < n; i += 32) {
        cd v;
        if (i == j) { v.re = 1; v.im = 0; } else v = W[i + (size_t)j * n];
        cd w = W[i + (size_t)c * n];
        w.re -= v.re * fr - v.im * fi;
        w.im -= v.re * fi + v.im * fr;
        W[i + (size_t)c * n] = w;
      }
    }
    __syncthreads();
  }
  // Vp = [0; I]
  const int q = n - k;
  for (int idx = threadIdx.x; idx < n * q; idx += NT) {
    const int r = idx % n, c = idx / n;
    cd v;
    v.re = (r == k + c) ? 1.0 : 0.0;
    v.im = 0;
    Vp[idx] = v;
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double tr = tau_r[j], ti = tau_i[j];
    if (tr == 0.0 && ti == 0.0) continue;
    for (int c = warp; c < q; c += nw) {
      double dr = 0, di = 0;
      for (int i = j + lane; i < n; i += 32) {
        const cd w = Vp[i + (size_t)c * n];
        cd v;
        if (i == j) { v.re = 1; v.im = 0; } else v = W[i + (size_t)j * n];
        dr += v.re * w.re + v.im * w.im;
        di += v.re * w.im - v.im * w.re;
      }
      dr = warp_sum(dr);
      di = warp_sum(di);
      const double fr = tr * dr - ti * di, fi = tr * di + ti * dr;  // tau * d
      for (int i = j + lane; i < n; i += 32) {
        cd v;
        if (i == j) { v.re = 1; v.im = 0; } else v = W[i + (size_t)j * n];
        cd w = Vp[i + (size_t)c * n];
        w.re -= v.re * fr - v.im * fi;
        w.im -= v.re * fi + v.im * fr;
        Vp[i + (size_t)c * n] = w;
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// Cyclic Jacobi for a Hermitian matrix with the parallel round-robin order:
// in each round the p/2 disjoint pairs rotate at once (columns of A and U,
// then rows of A).  A 2 x 2 Hermitian [[a, b],[conj b, d]] with b = g e^{i phi}
// is diagonalised by G = diag(1, e^{-i phi}) J, J the real symmetric Jacobi
// rotation of [[a, g],[g, d]] (tau = (d - a) / (2 g)).
__global__ void __launch_bounds__(NT) k_jacobi(const EigTask* __restrict__ tasks, int* status) {
  extern __shared__ double sh[];
  const EigTask t = tasks[blockIdx.x];
  const int p = t.p;
  if (p <= 0) return;
  const int pe = p + (p & 1);
  const int np = pe / 2;
  double* rc = sh;          // c per pair
  double* rs = rc + np;     // s
  double* rer = rs + np;    // e^{i phi} re
  double* rei = rer + np;   // e^{i phi} im
  int* pa = (int*)(rei + np);
  int* pb = pa + np;
  __shared__ double red[32];
  __shared__ int any_rot;
  cd* A = t.A;
  cd* U = t.U;
  for (int idx = threadIdx.x; idx < p * p; idx += NT) {
    cd v;
    v.re = (idx % p == idx / p) ? 1.0 : 0.0;
    v.im = 0;
    U[idx] = v;
  }
  __syncthreads();
  double fro = 0;
  for (int idx = threadIdx.x; idx < p * p; idx += NT) fro += A[idx].re * A[idx].re + A[idx].im * A[idx].im;
  fro = block_sum(fro, red);
  // rotations whose off-diagonal entry is below 4e-16 ||A||_F (or 1e-17 of
  // the geometric mean of the two diagonal entries) are skipped; the sweep
  // loop ends when a sweep would rotate nothing.
  // entries at the rounding level of the matrix are not rotated, nor entries
  // far below the truncation threshold of the rank decision (eq. 17), whose
  // rotation would move the eigenvalues by less than that floor
  const double gmin = fmax(fmax(1e-300, 4e-16 * sqrt(fro)), t.trM ? t.tol_rel * t.eps2 * (t.snorm2 + *t.trM) : 0.0);
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) any_rot = 0;
    __syncthreads();
    if (fro == 0.0) break;
    // converged when no off-diagonal entry is above its rotation threshold
    // (such a sweep would rotate nothing): one pass replaces that sweep
    {
      int any = 0;
      for (int idx = threadIdx.x; idx < p * p && !any; idx += NT) {
        const int row = idx % p, col = idx / p;
        if (row >= col) continue;
        const cd v = A[row + (size_t)col * p];
        const double g = sqrt(v.re * v.re + v.im * v.im);
        if (g > gmin && g > 1e-17 * sqrt(fabs(A[row + (size_t)row * p].re * A[col + (size_t)col * p].re))) any = 1;
      }
      if (!__syncthreads_or(any)) break;
    }
    for (int r = 0; r < pe - 1; ++r) {
      for (int i = threadIdx.x; i < np; i += NT) {
        int a, b;
        if (i == 0) { a = pe - 1; b = r; } else { a = (r + i) % (pe - 1); b = (r - i + pe - 1) % (pe - 1); }
        if (a > b) { const int x = a; a = b; b = x; }
        pa[i] = a;
        pb[i] = b;
        double c = 1, s = 0, er = 1, ei = 0;
        if (b < p) {
          const double app = A[a + (size_t)a * p].re, aqq = A[b + (size_t)b * p].re;
          const cd apq = A[a + (size_t)b * p];
          const double g2 = apq.re * apq.re + apq.im * apq.im;
          const double g = sqrt(g2);  // the threshold test of the convergence check
          const double rg = g2 > 0.0 ? rsqrt(g2) : 0.0;  // 1/g, issued beside the test
          if (g > gmin && g > 1e-17 * sqrt(fabs(app * aqq))) {
            any_rot = 1;
            er = apq.re * rg;
            ei = apq.im * rg;
            const double zeta = (aqq - app) * 0.5 * rg;
            const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = rsqrt(1.0 + tt * tt);
            s = tt * c;
          }
        }
        rc[i] = c;
        rs[i] = s;
        rer[i] = er;
        rei[i] = ei;
      }
      __syncthreads();
      // columns: A[:, a], A[:, b] and U[:, a], U[:, b]
      //   new a = c x_a - s conj(e) x_b ; new b = s x_a + c conj(e) x_b
      for (int idx = threadIdx.x; idx < np * p; idx += NT) {
        const int i = idx / p, row = idx % p;
        const double s = rs[i];
        if (s == 0.0) continue;
        const int a = pa[i], b = pb[i];
        const double c = rc[i], er = rer[i], ei = -rei[i];  // conj(e)
        for (int m = 0; m < 2; ++m) {
          cd* M = m == 0 ? A : U;
          const cd xa = M[row + (size_t)a * p], xb = M[row + (size_t)b * p];
          const double ebr = er * xb.re - ei * xb.im, ebi = er * xb.im + ei * xb.re;
          cd na, nb;
          na.re = c * xa.re - s * ebr;
          na.im = c * xa.im - s * ebi;
          nb.re = s * xa.re + c * ebr;
          nb.im = s * xa.im + c * ebi;
          M[row + (size_t)a * p] = na;
          M[row + (size_t)b * p] = nb;
        }
      }
      __syncthreads();
      // rows: new a = c y_a - s e y_b ; new b = s y_a + c e y_b
      for (int idx = threadIdx.x; idx < np * p; idx += NT) {
        const int i = idx / p, col = idx % p;
        const double s = rs[i];
        if (s == 0.0) continue;
        const int a = pa[i], b = pb[i];
        const double c = rc[i], er = rer[i], ei = rei[i];
        const cd ya = A[a + (size_t)col * p], yb = A[b + (size_t)col * p];
        const double ebr = er * yb.re - ei * yb.im, ebi = er * yb.im + ei * yb.re;
        cd na, nb;
        na.re = c * ya.re - s * ebr;
        na.im = c * ya.im - s * ebi;
        nb.re = s * ya.re + c * ebr;
        nb.im = s * ya.im + c * ebi;
        A[a + (size_t)col * p] = na;
        A[b + (size_t)col * p] = nb;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < np; i += NT) {
        if (rs[i] == 0.0) continue;
        const int a = pa[i], b = pb[i];
        cd z;
        z.re = 0;
        z.im = 0;
        A[a + (size_t)b * p] = z;
        A[b + (size_t)a * p] = z;
        A[a + (size_t)a * p].im = 0;
        A[b + (size_t)b * p].im = 0;
      }
      __syncthreads();
    }
    if (!any_rot) break;
  }
  if (sweep == kMaxSweeps && threadIdx.x == 0 && status) atomicMax(status, 2);
  if (threadIdx.x == 0 && t.sweeps) *t.sweeps = sweep;
  // sort eigenvalues in decreasing order (ties: lower index first); the
  // rank of each eigenvalue goes to shared memory (pa/pb hold >= p ints)
  int* rks = pa;
  for (int i = threadIdx.x; i < p; i += NT) {
    const double li = A[i + (size_t)i * p].re;
    int rank = 0;
    for (int j = 0; j < p; ++j) {
      const double lj = A[j + (size_t)j * p].re;
      rank += (lj > li) || (lj == li && j < i);
    }
    rks[i] = rank;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += NT) t.lam[rks[i]] = A[i + (size_t)i * p].re;
  __syncthreads();
  // A is free now: copy U there and write the columns back permuted
  for (int idx = threadIdx.x; idx < p * p; idx += NT) A[idx] = U[idx];
  __syncthreads();
  for (int idx = threadIdx.x; idx < p * p; idx += NT) {
    const int row = idx % p, col = idx / p;
    U[row + (size_t)rks[col] * p] = A[idx];
  }
}

// ----------------------------------------------------------------------------
// Partial-pivoting LU of an m x m block (in place, ld lda), pivot = largest
// |z| in the column, ties -> lowest row; then L^{-1} P and U^{-1}.

// ----------------------------------------------------------------------------
template <class ES, class ED>
__device__ __forceinline__ void cvt(const ES& s, ED& d, double al) {
  d.re = (decltype(d.re))(al * (double)s.re);
  d.im = (decltype(d.im))(al * (double)s.im);
}

// Work unit: 32 consecutive rows of one column (lane = row), units dealt to
// the task's warps; each warp takes CU units at a time with all their loads
// issued before any store (the destination may not alias the source, except
// in accumulate mode where it is read first).
template <class ES, class ED>
__device__ void copy_body(const CopyTask& t) {
  constexpr int CU = 4;
  const ES* S = (const ES*)t.src;
  ED* D = (ED*)t.dst;
  if (t.rows <= 0 || t.cols <= 0) return;
  const int nrb = (t.rows + 31) >> 5;
  const int units = nrb * t.cols;
  const int lane = threadIdx.x & 31;
  const int nw = (NT / 32) * gridDim.y;
  const int gw = (threadIdx.x >> 5) + blockIdx.y * (NT / 32);
  for (int u0 = gw; u0 < units; u0 += nw * CU) {
    ES sv[CU];
    ED ov[CU];
    int rr[CU], cc[CU];
    unsigned st = 0;  // per unit: bit 0 in range, bit 1 loaded from S
#pragma unroll
    for (int k = 0; k < CU; ++k) {
      const int u = u0 + k * nw;
      const int c = u / nrb, r = (u - c * nrb) * 32 + lane;
      rr[k] = r;
      cc[k] = c;
      if (u >= units || r >= t.rows) continue;
      st |= 1u << (2 * k);
      if (t.mode != 2 && S && r < t.srows && c < t.scols) {
        sv[k] = t.transpose ? S[(size_t)c + (size_t)r * t.lds] : S[(size_t)r + (size_t)c * t.lds];
        st |= 2u << (2 * k);
      }
      if (t.mode == 1) ov[k] = D[(size_t)r + (size_t)c * t.ldd];
    }
#pragma unroll
    for (int k = 0; k < CU; ++k) {
      if (!((st >> (2 * k)) & 1u)) continue;
      const int r = rr[k], c = cc[k];
      ED v;
      if (t.mode == 2) {
        v.re = (r == c) ? 1 : 0;
        v.im = 0;
      } else if ((st >> (2 * k)) & 2u) {
        cvt(sv[k], v, t.alpha);
      } else {
        v.re = 0;
        v.im = 0;
      }
      if (t.mode == 1) {
        v.re += ov[k].re;
        v.im += ov[k].im;
      }
      D[(size_t)r + (size_t)c * t.ldd] = v;
    }
  }
}

__global__ void __launch_bounds__(NT) k_copy2d(const CopyTask* __restrict__ tasks) {
  const CopyTask t = tasks[blockIdx.x];
  if (t.src_prec == P64 && t.dst_prec == P64) copy_body<cd, cd>(t);
  else if (t.src_prec == P64 && t.dst_prec == P32) copy_body<cd, cf>(t);
  else if (t.src_prec == P32 && t.dst_prec == P64) copy_body<cf, cd>(t);
  else copy_body<cf, cf>(t);
}

template <class EI, class EO>
__global__ void k_permute_scale(const EI* in, EO* out, const int64_t* perm, const double* scale, int64_t N,
                                int nrhs, int inverse, int conj) {
  const int64_t tot = N * (int64_t)nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx % N, c = idx / N;
    const int64_t g = perm ? perm[p] : p;
    const double sc = scale ? scale[g] : 1.0;
    if (!inverse) {
      // out (tree order) <- in (global order)
      const EI v = in[g + c * N];
      EO o;
      o.re = (decltype(o.re))(sc * (double)v.re);
      o.im = (decltype(o.im))(sc * (conj ? -(double)v.im : (double)v.im));
      out[p + c * N] = o;
    } else {
      // out (global order) <- in (tree order)
      const EI v = in[p + c * N];
      EO o;
      o.re = (decltype(o.re))(sc * (double)v.re);
      o.im = (decltype(o.im))(sc * (conj ? -(double)v.im : (double)v.im));
      out[g + c * N] = o;
    }
  }
}

__global__ void k_col_norms2(const cd* x, int64_t N, double* out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0;
  for (int64_t i = threadIdx.x; i < N; i += NT) {
    const cd v = x[i + (int64_t)c * N];
    s += v.re * v.re + v.im * v.im;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[c] = s;
}

// ||block||_F^2 of every block (one CTA per block), then per task the sum of
// its blocks' partials in block order (deterministic)
template <class E>
__global__ void k_frob2_part(const FrobBlock* __restrict__ blocks, double* __restrict__ part) {
  __shared__ double red[32];
  const FrobBlock k = blocks[blockIdx.x];
  const E* A = (const E*)k.A;
  double s = 0;
  // one warp per column, lanes over its rows (coalesced, no index division)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < k.cols; c += NT / 32) {
    const E* col = A + (int64_t)c * k.lda;
    for (int r = lane; r < k.rows; r += 32) {
      const E v = col[r];
      s += (double)v.re * (double)v.re + (double)v.im * (double)v.im;
    }
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_frob2_sum(const FrobTask* __restrict__ tasks, int ntasks, const double* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntasks) return;
  const FrobTask t = tasks[i];
  double s = 0;
  for (int b = t.b0; b < t.b0 + t.nb; ++b) s += part[b];
  *t.out = s;
}

__global__ void k_axpby(const cd* a, const cd* b, cd* y, int64_t n, double al, double be) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cd v;
    v.re = al * a[i].re + be * b[i].re;
    v.im = al * a[i].im + be * b[i].im;
    y[i] = v;
  }
}

template <class EI, class EO>
__global__ void k_convert(const EI* in, EO* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    EO o;
    o.re = (decltype(o.re))in[i].re;
    o.im = (decltype(o.im))in[i].im;
    out[i] = o;
  }
}

template <class E>
__global__ void k_set_diag(E* A, int lda, int n, double v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    E e;
    e.re = (decltype(e.re))v;
    e.im = 0;
    A[(size_t)i + (size_t)i * lda] = e;
  }
}

inline int grid_for(int64_t n) {
  int64_t g = (n + NT - 1) / NT;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t householder_complement(const HhTask* d, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_householder<<<n, NT, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t jacobi_eig(const EigTask* d, int n, int maxp, int* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int np = (maxp + 1) / 2 + 1;
  size_t sm = (size_t)np * (4 * sizeof(double) + 2 * sizeof(int));
  if (sm < (size_t)maxp * sizeof(int) + 64) sm = (size_t)maxp * sizeof(int) + 64;
  k_jacobi<<<n, NT, sm, s>>>(d, st);
  return cudaGetLastError();
}

cudaError_t set_diag(void* A, int lda, int n, int prec, double v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (prec == P64) k_set_diag<cd><<<grid_for(n), NT, 0, s>>>((cd*)A, lda, n, v);
  else k_set_diag<cf><<<grid_for(n), NT, 0, s>>>((cf*)A, lda, n, v);
  return cudaGetLastError();
}

cudaError_t copy2d(const CopyTask* d, int n, cudaStream_t s, int ctas_per_task) {
  if (n <= 0) return cudaSuccess;
  k_copy2d<<<dim3(n, std::max(1, std::min(32, ctas_per_task))), NT, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t permute_scale(const void* in, void* out, const int64_t* perm, const double* scale, int64_t N,
                          int nrhs, int ip, int op, int inverse, int conj, cudaStream_t s) {
  const int g = grid_for(N * nrhs);
  if (ip == P64 && op == P64)
    k_permute_scale<cd, cd><<<g, NT, 0, s>>>((const cd*)in, (cd*)out, perm, scale, N, nrhs, inverse, conj);
  else if (ip == P64 && op == P32)
    k_permute_scale<cd, cf><<<g, NT, 0, s>>>((const cd*)in, (cf*)out, perm, scale, N, nrhs, inverse, conj);
  else if (ip == P32 && op == P64)
    k_permute_scale<cf, cd><<<g, NT, 0, s>>>((const cf*)in, (cd*)out, perm, scale, N, nrhs, inverse, conj);
  else
    k_permute_scale<cf, cf><<<g, NT, 0, s>>>((const cf*)in, (cf*)out, perm, scale, N, nrhs, inverse, conj);
  return cudaGetLastError();
}

cudaError_t col_norms2(const cd* x, int64_t N, int nrhs, double* out, cudaStream_t s) {
  if (nrhs <= 0) return cudaSuccess;
  k_col_norms2<<<nrhs, NT, 0, s>>>(x, N, out);
  return cudaGetLastError();
}

cudaError_t frob2(const FrobTask* d_tasks, int ntasks, const FrobBlock* d_blocks, int nblocks, double* d_part,
                  int prec, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (nblocks > 0) {
    if (prec == P64) k_frob2_part<cd><<<nblocks, NT, 0, s>>>(d_blocks, d_part);
    else k_frob2_part<cf><<<nblocks, NT, 0, s>>>(d_blocks, d_part);
  }
  k_frob2_sum<<<(ntasks + 127) / 128, 128, 0, s>>>(d_tasks, ntasks, d_part);
  return cudaGetLastError();
}

cudaError_t axpby(const cd* a, const cd* b, cd* y, int64_t n, double al, double be, cudaStream_t s) {
  k_axpby<<<grid_for(n), NT, 0, s>>>(a, b, y, n, al, be);
  return cudaGetLastError();
}

cudaError_t convert(const void* in, int ip, void* out, int op, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (ip == P64 && op == P32) k_convert<cd, cf><<<grid_for(n), NT, 0, s>>>((const cd*)in, (cf*)out, n);
  else if (ip == P32 && op == P64) k_convert<cf, cd><<<grid_for(n), NT, 0, s>>>((const cf*)in, (cd*)out, n);
  else if (ip == P64 && op == P64) k_convert<cd, cd><<<grid_for(n), NT, 0, s>>>((const cd*)in, (cd*)out, n);
  else k_convert<cf, cf><<<grid_for(n), NT, 0, s>>>((const cf*)in, (cf*)out, n);
  return cudaGetLastError();
}

}  // namespace h2k
