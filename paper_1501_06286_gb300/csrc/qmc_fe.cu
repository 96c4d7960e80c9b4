// qmc_fe.cu — the finite-element step after the product in Sections 3.2 and
// 3.3 (Experiments 2 and 3): for every QMC point y_n, the symmetric
// tridiagonal stiffness matrix B(y_n) of the hat functions φ_k, k = 1..M-1,
// the solve B(y_n) û^(n) = ĝ, and the mean ū = (1/N) Σ_n û^(n).
//
// The stiffness condition number grows like M^2 (about 2.6e7 at M = 8002),
// beyond an FP32 solve at the 1e-5 target, so the solve is FP64; and one
// serial elimination per system leaves the GPU idle (4001 systems are 126
// warps).  So each system is solved by a block of 128 threads with a
// partitioned elimination: chunks of the unknowns eliminated in parallel,
// their interface values from a small tridiagonal system, then back
// substitution (k_fe_spike).  A second kernel takes the mean over the
// systems of each û_k in a fixed order (deterministic).
#include "qmc_internal.h"

namespace qmc {

namespace {

// 1/x in FP64 by Newton's iteration r <- r + r(1 - x r) from the FP32
// reciprocal of x (each step squares the relative error: two steps reach
// FP64 rounding); x must lie inside FP32's normal range, which the
// power-of-two scaling of each system provides.
__device__ __forceinline__ double recip64(double x) {
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// ---------------------------------------------------------------------------
// Partitioned solve, one block of kFeChunks threads per system.  The K =
// M - 1 unknowns split into chunks of C rows (thread c owns rows
// [c·C, c·C + C)); the last row of every chunk but the last is an
// interface unknown z_c.  With the interfaces fixed, the other rows of a
// chunk (its interior, rows lo..L) form a tridiagonal system whose solution
// is
//   x = y - z_{c-1} w - z_c v,   A y = ĝ,  A w = E_{lo-1} e_first,  A v = E_L e_last,
// so the interface rows give a tridiagonal system in the z_c alone:
//   -E_{h-1} w_L z_{c-1} + (D_h - E_{h-1} v_L - E_h w'_F) z_c - E_h v'_F z_{c+1}
//     = ĝ_h - E_{h-1} y_L - E_h y'_F
// (h the interface row, L / F the last / first interior rows of the chunks
// on either side, primes for chunk c+1).  Phase 1: each thread eliminates
// its interior top-down, storing the modified c', y', w' (their last values
// are y_L, w_L and v_L = E_L / pivot_L), then runs the back substitution of
// y, w and v to their first values.  Thread 0 solves the interface system.
// Phase 2: back substitution of the interior with the z_c known; the
// solution is stored over c'.  Everything is FP64; each system is first
// scaled by a power of two (exact), so that the pivots stay inside the FP32
// range the reciprocal's starting value needs.
// ---------------------------------------------------------------------------
constexpr int kFeChunks = 128;   // chunks (threads) per system
constexpr int kFeMinChunk = 8;   // rows per chunk at least

__host__ __device__ inline int fe_chunk_rows(int K) {
  const int c = (K + kFeChunks - 1) / kFeChunks;
  return c < kFeMinChunk ? kFeMinChunk : c;
}

__global__ void __launch_bounds__(kFeChunks) k_fe_spike(const float* __restrict__ B, int64_t ldb, int M, int kind,
                                                          const double* __restrict__ g_hat, double* __restrict__ work) {
  const int K = M - 1;
  const int C = fe_chunk_rows(K);
  const int nch = (K + C - 1) / C;
  const int c = threadIdx.x;
  const int64_t n = blockIdx.x;
  const float* row = B + n * ldb;
  const bool mid = kind == QMC_FE_MIDPOINT;
  const int64_t region = (int64_t)3 * C * kFeChunks;  // doubles per system: c', y', w'
  double* CP = work + n * region;
  double* YP = CP + (int64_t)C * kFeChunks;
  double* WP = YP + (int64_t)C * kFeChunks;
  auto slot = [&](int k, int lo) { return (int64_t)(k - lo) * kFeChunks + c; };

  __shared__ float s_max[kFeChunks / 32];
  __shared__ double yL[kFeChunks], wL[kFeChunks], vL[kFeChunks], yF[kFeChunks], wF[kFeChunks], vF[kFeChunks];
  __shared__ double zs[kFeChunks];

  const int lo = c * C;
  const bool active = c < nch;
  const int hi = active ? min(K, lo + C) - 1 : lo;
  const bool last = c == nch - 1;
  const int L = last ? hi : hi - 1;  // last interior row

  // scale 2^-e from the largest coefficient magnitude of the row
  float mx = 0.f;
  if (active) {
    const int top = mid ? (last ? K : hi) : hi;
    for (int k = lo; k <= top; ++k) mx = fmaxf(mx, fabsf(row[k]));
    if (!mid)
      for (int k = lo; k <= hi && k <= K - 2; ++k) mx = fmaxf(mx, fabsf(row[K + k]));
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((c & 31) == 0) s_max[c >> 5] = mx;
  __syncthreads();
  mx = fmaxf(fmaxf(s_max[0], s_max[1]), fmaxf(s_max[2], s_max[3]));
  if (mid) mx *= 2.f * (float)M;
  const int ex = mx > 0.f ? ilogbf(mx) : 0;
  const double sc = ldexp(1.0, -ex);               // exact power of two
  const double msc = mid ? (double)M * sc : sc;

  // scaled coefficients (exact in FP64)
  auto Dk = [&](int k) -> double {
    return mid ? ((double)row[k] + (double)row[k + 1]) * msc : (double)row[k] * sc;
  };
  auto Ek = [&](int k) -> double {  // b_{k,k+1}; zero outside 0..K-2
    if (k < 0 || k > K - 2) return 0.0;
    return mid ? -(double)row[k + 1] * msc : (double)row[K + k] * sc;
  };
  auto gk = [&](int k) -> double { return g_hat ? g_hat[k] : 1.0; };

  double vLast = 0.0;  // v'_L = E_L / pivot_L
  if (active) {
    // top-down elimination of the interior, storing c', y', w'
    double cp = 0.0, yp = 0.0, wp = 0.0, r = 0.0;
    double Eprev = Ek(lo - 1);
    for (int k = lo; k <= L; ++k) {
      const double E = Ek(k);
      r = recip64(Dk(k) - Eprev * cp);   // cp = 0 at k = lo
      cp = E * r;
      yp = (gk(k) - Eprev * yp) * r;     // yp = 0 at k = lo
      wp = k == lo ? Eprev * r : -Eprev * wp * r;
      CP[slot(k, lo)] = cp;
      YP[slot(k, lo)] = yp;
      WP[slot(k, lo)] = wp;
      Eprev = E;
    }
    vLast = Ek(L) * r;
    yL[c] = yp;
    wL[c] = wp;
    vL[c] = vLast;
    // back substitution of y, w, v to the first interior row
    double y = yp, w = wp, v = vLast;
    for (int k = L - 1; k >= lo; --k) {
      const double cc = CP[slot(k, lo)];
      y = YP[slot(k, lo)] - cc * y;
      w = WP[slot(k, lo)] - cc * w;
      v = -cc * v;
    }
    yF[c] = y;
    wF[c] = w;
    vF[c] = v;
  }
  __syncthreads();

  // interface system (nch - 1 unknowns), Thomas by thread 0
  if (c == 0) {
    const int nif = nch - 1;
    double cprev = 0.0, dprev = 0.0;
    for (int q = 0; q < nif; ++q) {
      const int h = (q + 1) * C - 1;
      const double Em = Ek(h - 1), Eh = Ek(h);
      const double al = -Em * wL[q];
      const double be = Dk(h) - Em * vL[q] - Eh * wF[q + 1];
      const double ga = -Eh * vF[q + 1];
      const double de = gk(h) - Em * yL[q] - Eh * yF[q + 1];
      const double rden = recip64(be - al * cprev);
      cprev = ga * rden;
      dprev = (de - al * dprev) * rden;
      yL[q] = cprev;  // reuse: modified c and d of the interface rows
      wL[q] = dprev;
    }
    double z = 0.0;
    for (int q = nif - 1; q >= 0; --q) {
      z = wL[q] - yL[q] * z;
      zs[q] = z;
    }
  }
  __syncthreads();

  // back substitution of the interior; x (scaled back) over c'
  if (active) {
    const double zp = c > 0 ? zs[c - 1] : 0.0;
    const double zn = last ? 0.0 : zs[c];
    double x = 0.0;
    for (int k = L; k >= lo; --k) {
      double d = YP[slot(k, lo)] - zp * WP[slot(k, lo)];
      if (k == L) d -= zn * vLast;
      x = k == L ? d : d - CP[slot(k, lo)] * x;
      CP[slot(k, lo)] = x * sc;
    }
    if (!last) CP[slot(hi, lo)] = zn * sc;
  }
}

// ū_k = (1/N) Σ_n x_k^(n).  A block takes 32 neighbouring positions p =
// i·kFeChunks + c of the stored solutions (row k = c·C + i); warp g of 8
// sums the systems n ≡ g (mod 8) in index order, and the 8 partial sums are
// added in warp order: a fixed order, so the result is deterministic.
__global__ void __launch_bounds__(256) k_fe_mean2(const double* __restrict__ work, int64_t n_sys, int M,
                                                   double* __restrict__ u_mean) {
  __shared__ double part[8][32];
  const int K = M - 1;
  const int C = fe_chunk_rows(K);
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  const int64_t region = (int64_t)3 * C * kFeChunks;
  double v = 0.0;
  if (p < C * kFeChunks) {
    for (int64_t n = g; n < n_sys; n += 8) v += work[n * region + p];
  }
  part[g][lane] = v;
  __syncthreads();
  if (g == 0 && p < C * kFeChunks) {
    const int i = p / kFeChunks, c = p % kFeChunks;
    const int k = c * C + i;
    if (k < K) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += part[q][lane];
      u_mean[k] = t / (double)n_sys;
    }
  }
}

}  // namespace

}  // namespace qmc

using namespace qmc;

extern "C" {

int64_t qmc_fe_work_bytes(int64_t n_sys, int32_t M) {
  if (n_sys < 1 || M < 3) return 0;
  // per system: c', y', w' for every chunk slot; the solution is written
  // over c'
  return n_sys * 3 * (int64_t)fe_chunk_rows(M - 1) * kFeChunks * (int64_t)sizeof(double);
}

int qmc_fe_solve_mean(const float* B, int64_t ldb, int64_t n_sys, int32_t M, int32_t kind, const double* g_hat,
                      void* work, int64_t work_bytes, double* u_mean, void* stream) {
  if (!B || !work || !u_mean || M < 3 || n_sys < 1 || (kind != QMC_FE_TRIDIAG && kind != QMC_FE_MIDPOINT) ||
      ((uintptr_t)work & 7u) != 0)
    return QMC_ERR_INVALID;
  const int64_t row_len = kind == QMC_FE_TRIDIAG ? 2 * (int64_t)M - 3 : (int64_t)M;
  if (ldb < row_len || work_bytes < qmc_fe_work_bytes(n_sys, M)) return QMC_ERR_SHAPE;
  if (n_sys > 0x7fffffff) return QMC_ERR_SHAPE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* w = static_cast<double*>(work);
  k_fe_spike<<<(unsigned)n_sys, kFeChunks, 0, st>>>(B, ldb, M, kind, g_hat, w);
  count_launch();
  const int slots = fe_chunk_rows(M - 1) * kFeChunks;
  k_fe_mean2<<<(slots + 31) / 32, 256, 0, st>>>(w, n_sys, M, u_mean);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // extern "C"
