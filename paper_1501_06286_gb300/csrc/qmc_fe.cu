// qmc_fe.cu — the finite-element step after the product in Sections 3.2 and
// 3.3 (Experiments 2 and 3): for every QMC point y_n, the symmetric
// tridiagonal stiffness matrix B(y_n) of the hat functions φ_k, k = 1..M-1,
// the solve B(y_n) û^(n) = ĝ, and the mean ū = (1/N) Σ_n û^(n).
//
// One thread per system, FP64 elimination without pivoting (the Thomas
// algorithm; the experiments' matrices are positive definite), its pivot
// reciprocals by Newton's iteration.  The
// stiffness condition number grows like M^2 (about 2.6e7 at M = 8002), too
// much for an FP32 solve at the 1e-5 target, so the solve is FP64 on the
// FP32 rows the product wrote.  Each thread eliminates its system from both
// ends towards the middle unknown (two independent pivot recurrences, half
// as long as one), reading its row of B eight steps ahead, keeps the
// eliminated coefficients in the work array k-major (a warp's threads store
// 32 consecutive doubles), then substitutes outwards from the middle (loads
// eight steps ahead) and writes û_k over them; a second kernel takes the
// mean over the systems of each û_k in a fixed order.
#include "qmc_internal.h"

namespace qmc {

namespace {

constexpr int kFeThreads = 32;  // one warp per block: the few systems spread over all SMs
constexpr int kFeUnroll = 8;    // steps whose loads are issued together

// 1/x in FP64 by Newton's iteration for the reciprocal, r <- r + r(1 - x r),
// which squares the relative error each step: from the FP32 approximate
// reciprocal (about 2^-23) two steps reach FP64 rounding.  The pivot
// recurrence of the solve runs through this reciprocal, so it is kept to
// one approximate FP32 operation and four FP64 FMAs.  The FP32 start needs
// x well inside FP32's normal range (the pivots here are about M times the
// coefficient); a pivot outside [1e-30, 1e30] in magnitude (or zero, or not
// finite) takes the FP64 division instead, so that an extreme row of B
// costs speed, not accuracy.
__device__ __forceinline__ double newton_recip(double x) {
  const double ax = fabs(x);
  if (!(ax >= 1e-30 && ax <= 1e30)) return 1.0 / x;
  float r32;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r32) : "f"((float)x));
  double r = (double)r32;
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

__global__ void k_fe_solve(const float* __restrict__ B, int64_t ldb, int64_t n_sys, int M, int kind,
                           const double* __restrict__ g_hat, double* __restrict__ cw, double* __restrict__ dw) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= n_sys) return;
  const int K = M - 1;       // unknowns û_1..û_{M-1} (0-based k below)
  const int m = K / 2;       // the middle unknown, where the two eliminations meet
  const int nb = K - 1 - m;  // steps of the bottom-up elimination (m of the top-down one)
  const float* row = B + n * ldb;
  const double dM = (double)M;
  const bool mid = kind == QMC_FE_MIDPOINT;
  constexpr int U = kFeUnroll;
  auto g = [&](int k) { return g_hat ? g_hat[k] : 1.0; };
  auto w = [&](int k) { return (int64_t)k * n_sys + n; };

  // Elimination from both ends (two independent recurrences, so the
  // thread's FP64 pivot chains overlap).  With D_k = b_kk, E_k = b_{k,k+1}:
  //   top-down, k = 0..m-1:    c'_k = E_k / p,      d'_k = (ĝ_k - E_{k-1} d'_{k-1}) / p,
  //                            p = D_k - E_{k-1} c'_{k-1};
  //   bottom-up, k = K-1..m+1: c''_k = E_{k-1} / p,  d''_k = (ĝ_k - E_k d''_{k+1}) / p,
  //                            p = D_k - E_k c''_{k+1}.
  // Midpoint rows: D_k = M (a_k + a_{k+1}), E_k = -M a_{k+1} (a = row).
  double ct = 0.0, dt = 0.0, et = 0.0;        // top: c'_{k-1}, d'_{k-1}, E_{k-1}
  double cb = 0.0, db = 0.0, eb = 0.0;        // bottom: c''_{k+1}, d''_{k+1}, E_k
  double at = mid ? (double)row[0] : 0.0;     // top: a_k (midpoint rows)
  double ab = mid ? (double)row[K] : 0.0;     // bottom: a_{k+1}
  for (int i0 = 0; i0 < m; i0 += U) {
    float xt[U], yt[U], xb[U], yb[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int i = i0 + q;
      const int k = i, kb = K - 1 - i;
      xt[q] = i < m ? row[mid ? k + 1 : k] : 0.f;              // a_{k+1} | D_k
      yt[q] = (!mid && i < m && k <= K - 2) ? row[K + k] : 0.f;  // E_k (tridiagonal rows)
      xb[q] = i < nb ? row[kb] : 0.f;                          // a_kb | D_kb
      yb[q] = (!mid && i < nb) ? row[K + kb - 1] : 0.f;        // E_{kb-1} (tridiagonal rows)
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int i = i0 + q;
      if (i >= m) break;
      {
        const int k = i;
        const double a1 = (double)xt[q];
        const double Dk = mid ? dM * (at + a1) : a1;
        const double Ek = mid ? (k <= K - 2 ? -dM * a1 : 0.0) : (double)yt[q];
        const double r = newton_recip(Dk - et * ct);
        const double c = Ek * r, d = (g(k) - et * dt) * r;
        cw[w(k)] = c;
        dw[w(k)] = d;
        ct = c; dt = d; et = Ek; at = a1;
      }
      if (i < nb) {
        const int k = K - 1 - i;
        const double a0 = (double)xb[q];
        const double Dk = mid ? dM * (a0 + ab) : a0;
        const double Em = mid ? -dM * a0 : (double)yb[q];  // E_{k-1}
        const double r = newton_recip(Dk - eb * cb);
        const double c = Em * r, d = (g(k) - eb * db) * r;
        cw[w(k)] = c;
        dw[w(k)] = d;
        cb = c; db = d; eb = Em; ab = a0;
      }
    }
  }
  // the middle unknown: row m with û_{m-1} = d'_{m-1} - c'_{m-1} û_m and
  // û_{m+1} = d''_{m+1} - c''_{m+1} û_m (et = E_{m-1}; eb = E_m when nb > 0)
  const double Dm = mid ? dM * ((double)row[m] + (double)row[m + 1]) : (double)row[m];
  double num = g(m) - et * dt, den = Dm - et * ct;
  if (nb > 0) {
    num -= eb * db;
    den -= eb * cb;
  }
  const double um = num / den;
  dw[w(m)] = um;

  // back substitution outwards from the middle, both directions at once,
  // loads U steps ahead; û_k is written over d'_k / d''_k
  double ut = um, ubt = um;
  for (int i0 = 0; i0 < m; i0 += U) {
    double c1[U], d1[U], c2[U], d2[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int i = i0 + q;
      const int k = m - 1 - i, kb = m + 1 + i;
      c1[q] = i < m ? cw[w(k)] : 0.0;
      d1[q] = i < m ? dw[w(k)] : 0.0;
      c2[q] = i < nb ? cw[w(kb)] : 0.0;
      d2[q] = i < nb ? dw[w(kb)] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int i = i0 + q;
      if (i >= m) break;
      ut = d1[q] - c1[q] * ut;
      dw[w(m - 1 - i)] = ut;
      if (i < nb) {
        ubt = d2[q] - c2[q] * ubt;
        dw[w(m + 1 + i)] = ubt;
      }
    }
  }
}

// ū_k = (1/N) Σ_n û_k^(n): one block per k, a fixed-order block sum of the
// n_sys contiguous values (deterministic).
__global__ void k_fe_mean(const double* __restrict__ dw, int64_t n_sys, double* __restrict__ u_mean) {
  __shared__ double part[32];
  const int k = blockIdx.x;
  const double* x = dw + (int64_t)k * n_sys;
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n_sys; i += blockDim.x) v += x[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) u_mean[k] = v / (double)n_sys;
  }
}

}  // namespace

}  // namespace qmc

using namespace qmc;

extern "C" {

int64_t qmc_fe_work_bytes(int64_t n_sys, int32_t M) {
  if (n_sys < 1 || M < 3) return 0;
  return 2 * (int64_t)(M - 1) * n_sys * (int64_t)sizeof(double);
}

int qmc_fe_solve_mean(const float* B, int64_t ldb, int64_t n_sys, int32_t M, int32_t kind, const double* g_hat,
                      void* work, int64_t work_bytes, double* u_mean, void* stream) {
  if (!B || !work || !u_mean || M < 3 || n_sys < 1 || (kind != QMC_FE_TRIDIAG && kind != QMC_FE_MIDPOINT) ||
      ((uintptr_t)work & 7u) != 0)
    return QMC_ERR_INVALID;
  const int64_t row_len = kind == QMC_FE_TRIDIAG ? 2 * (int64_t)M - 3 : (int64_t)M;
  if (ldb < row_len || work_bytes < qmc_fe_work_bytes(n_sys, M)) return QMC_ERR_SHAPE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int K = M - 1;
  double* cw = static_cast<double*>(work);
  double* dw = cw + (int64_t)K * n_sys;
  const int64_t blocks = (n_sys + kFeThreads - 1) / kFeThreads;
  k_fe_solve<<<(unsigned)blocks, kFeThreads, 0, st>>>(B, ldb, n_sys, M, kind, g_hat, cw, dw);
  count_launch();
  k_fe_mean<<<(unsigned)K, 256, 0, st>>>(dw, n_sys, u_mean);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // extern "C"
