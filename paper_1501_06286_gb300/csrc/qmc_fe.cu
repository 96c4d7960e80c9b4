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
// FP32 rows the product wrote.  Each thread reads its row of B left to
// right, eight entries ahead of the recurrence, keeps the modified
// super-diagonal c'_k and right-hand side d'_k in the work array k-major (a
// warp's threads store 32 consecutive doubles), then substitutes backwards
// (loads eight steps ahead) and writes û_k over d'_k; a second kernel takes
// the mean over the systems of each û_k in a fixed order.
#include "qmc_internal.h"

namespace qmc {

namespace {

constexpr int kFeThreads = 32;  // one warp per block: the few systems spread over all SMs
constexpr int kFeUnroll = 8;    // steps whose loads are issued together

// 1/x in FP64 by Newton's iteration for the reciprocal, r <- r + r(1 - x r),
// which squares the relative error each step: from the FP32 approximate
// reciprocal (about 2^-23) two steps reach FP64 rounding.  The pivot
// recurrence of the solve runs through this reciprocal, so it is kept to
// one approximate FP32 operation and four FP64 FMAs.  x must be a normal
// FP32-range number (the pivots here are about M times the coefficient).
__device__ __forceinline__ double newton_recip(double x) {
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
  const int K = M - 1;  // unknowns û_1..û_{M-1} (0-based k below)
  const float* row = B + n * ldb;
  const double dM = (double)M;
  constexpr int U = kFeUnroll;

  // forward elimination: den_k = b_kk - b_{k-1,k} c'_{k-1},
  // c'_k = b_{k,k+1} / den_k, d'_k = (ĝ_k - b_{k-1,k} d'_{k-1}) / den_k.
  // The row is read U entries ahead of the recurrence, whose FP64
  // reciprocal is the critical path.
  double c_prev = 0.0, d_prev = 0.0, e_prev = 0.0;
  for (int k0 = 0; k0 < K; k0 += U) {
    float dv[U], ev[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int k = k0 + q;
      if (kind == QMC_FE_MIDPOINT) {
        // node k+1 (1-based) lies on elements k+1 and k+2, whose midpoint
        // coefficients are row[k] and row[k+1]
        dv[q] = k < K ? row[k] : 0.f;
        ev[q] = k < K ? row[k + 1] : 0.f;
      } else {
        dv[q] = k < K ? row[k] : 0.f;
        ev[q] = k < K - 1 ? row[K + k] : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int k = k0 + q;
      if (k >= K) break;
      double dk, ek;
      if (kind == QMC_FE_MIDPOINT) {
        dk = dM * ((double)dv[q] + (double)ev[q]);     // b_{k,k} = M (a_k + a_{k+1})
        ek = k < K - 1 ? -dM * (double)ev[q] : 0.0;    // b_{k,k+1} = -M a_{k+1}
      } else {
        dk = (double)dv[q];
        ek = (double)ev[q];
      }
      const double r = newton_recip(dk - e_prev * c_prev);
      const double g = g_hat ? g_hat[k] : 1.0;
      const double ck = ek * r;
      const double dd = (g - e_prev * d_prev) * r;
      cw[(int64_t)k * n_sys + n] = ck;
      dw[(int64_t)k * n_sys + n] = dd;
      c_prev = ck;
      d_prev = dd;
      e_prev = ek;
    }
  }

  // back substitution, û_k = d'_k - c'_k û_{k+1}, written over d'_k; the
  // c'_k, d'_k of the next U steps are loaded before they are used
  double u = d_prev;  // û_{K-1} = d'_{K-1}
  for (int k0 = K - 2; k0 >= 0; k0 -= U) {
    double cv[U], dv[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int k = k0 - q;
      cv[q] = k >= 0 ? cw[(int64_t)k * n_sys + n] : 0.0;
      dv[q] = k >= 0 ? dw[(int64_t)k * n_sys + n] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int k = k0 - q;
      if (k < 0) break;
      u = dv[q] - cv[q] * u;
      dw[(int64_t)k * n_sys + n] = u;
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
