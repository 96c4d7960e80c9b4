// qmc_fe.cu — the finite-element step after the product in Sections 3.2 and
// 3.3 (Experiments 2 and 3): for every QMC point y_n, the symmetric
// tridiagonal stiffness matrix B(y_n) of the hat functions φ_k, k = 1..M-1,
// the solve B(y_n) û^(n) = ĝ, and the mean ū = (1/N) Σ_n û^(n).
//
// The stiffness condition number grows like M^2 (about 2.6e7 at M = 8002),
// beyond an FP32 solve at the 1e-5 target, so the solve is FP64; and one
// serial elimination per system leaves the GPU idle (4001 systems are 126
// warps).  So a general tridiagonal system (QMC_FE_TRIDIAG) is solved by a
// block of 128 threads with a partitioned elimination: chunks of the
// unknowns eliminated in parallel, their interface values from a small
// tridiagonal system, then back substitution (k_fe_spike); a second kernel
// takes the mean over the systems of each û_k in a fixed order.  The
// midpoint assembly (QMC_FE_MIDPOINT) has the element-difference form,
// whose solution and mean follow from sums (k_fe_flux_*, below), with no
// elimination at all.
#include "qmc_internal.h"

namespace qmc {

namespace {

// 1/x in FP64 from the FP32 reciprocal r of x (relative error e = 1 - x r,
// |e| <= 2^-24): 1/x = r / (1 - e) = r (1 + e + e^2 + ...), so
// r (1 + e + e^2) leaves an error of order e^3 (2^-72), below FP64
// rounding, in three FMAs (Newton's iteration, which only squares the
// error, needs two steps of two); x must lie inside FP32's normal range,
// which the power-of-two scaling of each system provides.
__device__ __forceinline__ double recip64(double x) {
  const double r = (double)__frcp_rn((float)x);
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
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

__global__ void __launch_bounds__(kFeChunks) k_fe_spike(const float* __restrict__ B, int64_t ldb, int M,
                                                          const double* __restrict__ g_hat, double* __restrict__ work) {
  const int K = M - 1;
  const int C = fe_chunk_rows(K);
  const int nch = (K + C - 1) / C;
  const int c = threadIdx.x;
  const int64_t n = blockIdx.x;
  const float* row = B + n * ldb;
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
    for (int k = lo; k <= hi; ++k) mx = fmaxf(mx, fabsf(row[k]));
    for (int k = lo; k <= hi && k <= K - 2; ++k) mx = fmaxf(mx, fabsf(row[K + k]));
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((c & 31) == 0) s_max[c >> 5] = mx;
  __syncthreads();
  mx = fmaxf(fmaxf(s_max[0], s_max[1]), fmaxf(s_max[2], s_max[3]));
  const int ex = mx > 0.f ? min(max(ilogbf(mx), -126), 126) : 0;
  const double sc = ldexp(1.0, -ex);               // exact power of two
  const float scf = ldexpf(1.0f, -ex);

  // scaled coefficients (the FP32 product by a power of two is exact for
  // every entry above 2^-126 times the row's largest)
  auto Dk = [&](int k) -> double { return (double)(row[k] * scf); };
  auto Ek = [&](int k) -> double {  // b_{k,k+1}; zero outside 0..K-2
    if (k < 0 || k > K - 2) return 0.0;
    return (double)(row[K + k] * scf);
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
      const double t = Eprev * r;        // E_{k-1} / pivot_k
      yp = fma(-t, yp, g_hat ? g_hat[k] * r : r);  // (ĝ_k - E_{k-1} y'_{k-1}) / pivot_k; yp = 0 at k = lo
      wp = k == lo ? t : -t * wp;
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


// ---------------------------------------------------------------------------
// Midpoint stiffness (QMC_FE_MIDPOINT) in flux form.  The assembled matrix
// is Dᵀ diag(M a) D, D the difference operator of the M elements (u_0 =
// u_M = 0).  With the element fluxes q_i = M a_i (u_i − u_{i−1}), row k of
// B(y) u = ĝ reads q_k − q_{k+1} = ĝ_k, so q_i = q_1 − G_{i−1} with
// G_j = ĝ_1 + … + ĝ_j, and u_k = (1/M) Σ_{i≤k} q_i r_i with r_i = 1/a_i;
// u_M = 0 fixes q_1 = Σ_i G_{i−1} r_i / Σ_i r_i.  The mean over the systems
// is then
//   ū_k = (1/(N M)) Σ_{i≤k} (Q_i − G_{i−1} S_i),
//   Q_i = Σ_n q_1^(n) r_i^(n),   S_i = Σ_n r_i^(n):
// two sums along each system's row (giving q_1), two column sums over the
// systems and one prefix sum, in place of N eliminations.  It is the same
// linear system's solution; only the order of the arithmetic differs.
//
// The row and column sums run in pairs of FP32 numbers (hi + lo, about 47
// significant bits; FP32 issues at 64 times the FP64 rate on this part):
// the reciprocals are formed as pairs from the correctly rounded FP32
// reciprocal and its residual 1 − a r, which the FMA gives exactly; a thread
// adds a few dozen terms before a fixed reduction tree.  Where Q_i − G S_i
// cancels, and in the prefix sum, the arithmetic is FP64.  Each system is
// scaled by a power of two (its largest coefficient into [1, 2)), and the
// right-hand side's prefix sums likewise, so that the pairs stay inside the
// FP32 range; a chunk of systems adds its column sums relative to its
// largest scale.  Sums over the same data are always taken in the same
// order (deterministic).
// ---------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfl df_norm(float hi, float lo) {  // |hi| >= |lo|
  const float s = __fadd_rn(hi, lo);
  return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  const dfl s = df_two_sum(x.hi, y.hi);
  return df_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_norm(p, e);
}
// 1/a as a pair (a > 0, normal): the hardware's approximate reciprocal r
// (within an ulp) and the Newton correction r (1 − a r), with the residual
// from one FMA: relative error about 2^-46
__device__ __forceinline__ dfl df_recip(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return {r, __fmul_rn(r, fmaf(-a, r, 1.0f))};
}
__device__ __forceinline__ double df_to_f64(dfl x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ dfl df_from_f64(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ dfl df_shfl_add(dfl x, int off) {
  dfl y;
  y.hi = __shfl_xor_sync(0xffffffffu, x.hi, off);
  y.lo = __shfl_xor_sync(0xffffffffu, x.lo, off);
  return df_add(x, y);
}

constexpr int kFluxChunk = 64;   // systems per column-sum chunk
constexpr int kFluxCols = 256;   // columns (elements) per column-sum block
constexpr int kScanThreads = 1024;

struct FluxSys {
  double q1;  // q_1 of the scaled system (scale-free)
  int ex;     // the system was scaled by 2^-ex
  int pad;
};

// Byte offsets of the flux solve's parts of the work buffer.
constexpr int kScanTile = 64;    // elements per block of the combination and the prefix sum

struct FluxLayout {
  int64_t hdr, gd, gdf, sys, qp, sp, r, tot, total;
  __host__ __device__ FluxLayout(int64_t n_sys, int M) {
    const int64_t nch = (n_sys + kFluxChunk - 1) / kFluxChunk;
    hdr = 0;
    gd = 64;
    gdf = gd + 8 * (int64_t)M;
    sys = gdf + 8 * (int64_t)M;
    qp = sys + 16 * n_sys;
    sp = qp + 8 * nch * M;
    r = sp + 8 * nch * M;
    tot = r + 8 * (int64_t)M;  // one sum of R per tile of kScanTile elements
    total = tot + 8 * (int64_t)((M + kScanTile - 1) / kScanTile);
  }
};

// Thread t of a kScanThreads block owns the segment [b, e) of 0..len.
__device__ __forceinline__ void scan_segment(int len, int& b, int& e) {
  const int seg = (len + kScanThreads - 1) / kScanThreads;
  b = min(len, (int)threadIdx.x * seg);
  e = min(len, b + seg);
}

// Exclusive prefix of the per-thread totals v over a kScanThreads block, in
// a fixed shape (warp scans, then a scan of the warp totals):
// deterministic.
__device__ double block_exclusive_prefix(double v, double* s_warp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double o = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += o;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    double w = s_warp[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double o = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += o;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const double before = wid > 0 ? s_warp[wid - 1] : 0.0;
  __syncthreads();
  const double excl = __shfl_up_sync(0xffffffffu, inc, 1);
  return lane > 0 ? before + excl : before;
}

// Prefix sums of the right-hand side, G_0 = 0, G_j = ĝ_1 + … + ĝ_j
// (j < M; ĝ ≡ 1 without g_hat), scaled by 2^-eg so that the largest is in
// [1, 2): FP64 (Gd) and as pairs (Gdf); 2^eg goes to the header.
__global__ void __launch_bounds__(kScanThreads) k_fe_flux_g(const double* __restrict__ g_hat, int M,
                                                             unsigned char* __restrict__ work) {
  __shared__ double s_warp[32];
  const FluxLayout lay(0, M);
  double* hdr = reinterpret_cast<double*>(work + lay.hdr);
  double* Gd = reinterpret_cast<double*>(work + lay.gd);
  dfl* Gdf = reinterpret_cast<dfl*>(work + lay.gdf);
  const int len = M - 1;
  int b, e;
  scan_segment(len, b, e);
  auto g = [&](int m) { return g_hat ? g_hat[m] : 1.0; };
  double tot = 0.0;
  for (int m = b; m < e; ++m) tot += g(m);
  const double run = block_exclusive_prefix(tot, s_warp);
  double x = run, mx = 0.0;
  for (int m = b; m < e; ++m) {
    x += g(m);
    mx = fmax(mx, fabs(x));
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int q = 0; q < kScanThreads / 32; ++q) mx = fmax(mx, s_warp[q]);
  const int eg = mx > 0.0 ? ilogb(mx) : 0;
  const double sc = ldexp(1.0, -eg);
  x = run;  // the same additions in the same order as above
  for (int m = b; m < e; ++m) {
    x += g(m);
    Gd[m + 1] = x * sc;
    Gdf[m + 1] = df_from_f64(x * sc);
  }
  if (threadIdx.x == 0) {
    Gd[0] = 0.0;
    Gdf[0] = dfl{0.f, 0.f};
    hdr[0] = ldexp(1.0, eg);
  }
}

// The same for ĝ ≡ 1: G_j = j, scaled by 2^-eg with eg = ilogb(M - 1);
// one thread per entry.
__global__ void __launch_bounds__(256) k_fe_flux_g_ones(int M, int eg, unsigned char* __restrict__ work) {
  const FluxLayout lay(0, M);
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= M) return;
  const float v = ldexpf((float)j, -eg);  // exact: j < 2^24
  reinterpret_cast<double*>(work + lay.gd)[j] = (double)v;
  reinterpret_cast<dfl*>(work + lay.gdf)[j] = dfl{v, 0.f};
  if (j == 0) reinterpret_cast<double*>(work + lay.hdr)[0] = ldexp(1.0, eg);
}

// Row sums of system n (one block of 256 threads): S = Σ_i r_i and
// T = Σ_i G_{i-1} r_i of the system scaled by 2^-ex, then q_1 = T / S.
__global__ void __launch_bounds__(256) k_fe_flux_rows(const float* __restrict__ B, int64_t ldb, int M,
                                                       unsigned char* __restrict__ work) {
  __shared__ float s_mx[8], s_mn[8];
  __shared__ dfl s_S[8], s_T[8];
  const int64_t n = blockIdx.x;
  const FluxLayout lay(0, M);
  const dfl* Gdf = reinterpret_cast<const dfl*>(work + lay.gdf);
  FluxSys* sys = reinterpret_cast<FluxSys*>(work + lay.sys);
  const float* row = B + n * ldb;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // one pass with the system unscaled (ex = 0), keeping its extreme
  // coefficients; a second, scaled pass only when they leave [2^-60, 2^60]
  float mx = 0.f, mn = 3.0e38f;
  dfl S{0.f, 0.f}, T{0.f, 0.f};
  for (int e = tid; e < M; e += 256) {
    const float a = row[e];
    mx = fmaxf(mx, a);
    mn = fminf(mn, a);
    const dfl r = df_recip(a);
    S = df_add(S, r);
    T = df_add(T, df_mul(Gdf[e], r));
  }
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
  }
  if (lane == 0) {
    s_mx[wid] = mx;
    s_mn[wid] = mn;
  }
  __syncthreads();
  mx = s_mx[0];
  mn = s_mn[0];
  for (int q = 1; q < 8; ++q) {
    mx = fmaxf(mx, s_mx[q]);
    mn = fminf(mn, s_mn[q]);
  }
  int ex = 0;
  if (!(mn >= 0x1p-60f && mx <= 0x1p60f)) {  // block-uniform
    ex = mx > 0.f ? min(max(ilogbf(mx), -126), 126) : 0;
    const float scf = ldexpf(1.0f, -ex);
    S = dfl{0.f, 0.f};
    T = dfl{0.f, 0.f};
    for (int e = tid; e < M; e += 256) {
      const dfl r = df_recip(row[e] * scf);
      S = df_add(S, r);
      T = df_add(T, df_mul(Gdf[e], r));
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    S = df_shfl_add(S, off);
    T = df_shfl_add(T, off);
  }
  if (lane == 0) {
    s_S[wid] = S;
    s_T[wid] = T;
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 1; q < 8; ++q) {
      S = df_add(S, s_S[q]);
      T = df_add(T, s_T[q]);
    }
    sys[n] = FluxSys{df_to_f64(T) / df_to_f64(S), ex, 0};
  }
}

// Column sums over a chunk of kFluxChunk systems, thread = element i:
// Q_i = Σ_n q_1^(n) r_i^(n) and S_i = Σ_n r_i^(n), each system's r taken
// relative to the chunk's largest scale 2^-E (E the smallest ex), written
// in FP64 at their true scale.  One block per (column tile, chunk).
__global__ void __launch_bounds__(kFluxCols) k_fe_flux_cols(const float* __restrict__ B, int64_t ldb, int M,
                                                             int64_t n_sys, unsigned char* __restrict__ work) {
  __shared__ float s_scf[kFluxChunk], s_wf[kFluxChunk];
  __shared__ dfl s_vq[kFluxChunk];
  __shared__ int s_ex[kFluxChunk];
  const FluxLayout lay(n_sys, M);
  const FluxSys* sys = reinterpret_cast<const FluxSys*>(work + lay.sys);
  double* Qp = reinterpret_cast<double*>(work + lay.qp);
  double* Sp = reinterpret_cast<double*>(work + lay.sp);
  const int ctiles = (M + kFluxCols - 1) / kFluxCols;
  const int64_t chunk = blockIdx.x / ctiles;
  const int e = (blockIdx.x % ctiles) * kFluxCols + threadIdx.x;
  const int64_t n0 = chunk * kFluxChunk;
  const int cnt = (int)min((int64_t)kFluxChunk, n_sys - n0);
  const int tid = threadIdx.x;
  if (tid < kFluxChunk) s_ex[tid] = tid < cnt ? sys[n0 + tid].ex : 0x7fffffff;
  __syncthreads();
  int E = s_ex[0];
  for (int q = 1; q < cnt; ++q) E = min(E, s_ex[q]);
  if (tid < cnt) {
    const int sh = E - s_ex[tid];  // <= 0
    s_scf[tid] = ldexpf(1.0f, -s_ex[tid]);
    s_wf[tid] = ldexpf(1.0f, sh);
    s_vq[tid] = df_from_f64(ldexp(sys[n0 + tid].q1, sh));
  }
  __syncthreads();
  if (e >= M) return;
  dfl Q{0.f, 0.f}, S{0.f, 0.f};
  const float* col = B + n0 * ldb + e;
#pragma unroll 4
  for (int j = 0; j < cnt; ++j) {
    const dfl r = df_recip(col[j * ldb] * s_scf[j]);
    Q = df_add(Q, df_mul(s_vq[j], r));
    const float w = s_wf[j];
    S = df_add(S, dfl{r.hi * w, r.lo * w});
  }
  Qp[chunk * M + e] = ldexp(df_to_f64(Q), -E);
  Sp[chunk * M + e] = ldexp(df_to_f64(S), -E);
}

// R_i = Q_i - G_{i-1} S_i for i = 1..M-1 (element e = i-1), the chunks'
// partial sums added in chunk order, FP64; and the sum of R over each tile
// of kScanTile elements (a fixed tree, deterministic).
__global__ void __launch_bounds__(kScanTile) k_fe_flux_combine(int M, int64_t n_sys, unsigned char* __restrict__ work) {
  __shared__ double s_w[kScanTile / 32];
  const FluxLayout lay(n_sys, M);
  const double* Gd = reinterpret_cast<const double*>(work + lay.gd);
  const double* Qp = reinterpret_cast<const double*>(work + lay.qp);
  const double* Sp = reinterpret_cast<const double*>(work + lay.sp);
  double* R = reinterpret_cast<double*>(work + lay.r);
  double* tot = reinterpret_cast<double*>(work + lay.tot);
  const int e = blockIdx.x * kScanTile + threadIdx.x;
  double v = 0.0;
  if (e < M - 1) {
    const int64_t nch = (n_sys + kFluxChunk - 1) / kFluxChunk;
    double Q = 0.0, S = 0.0;
#pragma unroll 8
    for (int64_t c = 0; c < nch; ++c) {
      Q += Qp[c * M + e];
      S += Sp[c * M + e];
    }
    v = fma(-Gd[e], S, Q);
    R[e] = v;
  }
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kScanTile / 32; ++q) t += s_w[q];
    tot[blockIdx.x] = t;
  }
}

// ū_k = 2^eg / (N M) · Σ_{e<k} R_e, k = 1..M-1 (u_mean[k-1]): the tiles
// before this one by their sums (in tile order), then a scan of the tile.
__global__ void __launch_bounds__(kScanTile) k_fe_flux_scan(int M, int64_t n_sys,
                                                            const unsigned char* __restrict__ work,
                                                            double* __restrict__ u_mean) {
  __shared__ double s_w[kScanTile / 32];
  __shared__ double s_off, s_scale;
  const FluxLayout lay(n_sys, M);
  const double* hdr = reinterpret_cast<const double*>(work + lay.hdr);
  const double* R = reinterpret_cast<const double*>(work + lay.r);
  const double* tot = reinterpret_cast<const double*>(work + lay.tot);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // offset: thread i adds tot[i], tot[i + kScanTile], ... below this tile,
  // then a fixed tree over the threads
  double o = 0.0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += kScanTile) o += tot[b];
  for (int off = 16; off > 0; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
  if (lane == 0) s_w[wid] = o;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kScanTile / 32; ++q) t += s_w[q];
    s_off = t;
    s_scale = hdr[0] / ((double)n_sys * (double)M);
  }
  __syncthreads();
  const int e = blockIdx.x * kScanTile + threadIdx.x;
  double inc = e < M - 1 ? R[e] : 0.0;
  for (int off = 1; off < 32; off <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += u;
  }
  __syncthreads();  // s_w is reused for the warp totals
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  double before = s_off;
  for (int q = 0; q < wid; ++q) before += s_w[q];
  if (e < M - 1) u_mean[e] = (before + inc) * s_scale;
}

}  // namespace

}  // namespace qmc

using namespace qmc;

extern "C" {

int64_t qmc_fe_work_bytes(int64_t n_sys, int32_t M) {
  if (n_sys < 1 || M < 3) return 0;
  // partitioned solve: per system, c', y', w' for every chunk slot (the
  // solution is written over c'); flux form: the layout of FluxLayout.
  // The larger of the two, so that one size serves both kinds.
  const int64_t spike = n_sys * 3 * (int64_t)fe_chunk_rows(M - 1) * kFeChunks * (int64_t)sizeof(double);
  const int64_t flux = FluxLayout(n_sys, M).total;
  return spike > flux ? spike : flux;
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
  if (kind == QMC_FE_MIDPOINT) {
    unsigned char* wb = static_cast<unsigned char*>(work);
    if (g_hat) {
      k_fe_flux_g<<<1, kScanThreads, 0, st>>>(g_hat, M, wb);
    } else {
      int eg = 0;
      while ((int64_t)2 << eg <= (int64_t)(M - 1)) ++eg;  // ilogb(M - 1)
      k_fe_flux_g_ones<<<(M + 255) / 256, 256, 0, st>>>(M, eg, wb);
    }
    count_launch();
    k_fe_flux_rows<<<(unsigned)n_sys, 256, 0, st>>>(B, ldb, M, wb);
    count_launch();
    const int64_t nch = (n_sys + kFluxChunk - 1) / kFluxChunk;
    const int64_t col_blocks = nch * ((M + kFluxCols - 1) / kFluxCols);
    if (col_blocks > 0x7fffffff) return QMC_ERR_SHAPE;
    k_fe_flux_cols<<<(unsigned)col_blocks, kFluxCols, 0, st>>>(B, ldb, M, n_sys, wb);
    count_launch();
    const int tiles = (M - 1 + kScanTile - 1) / kScanTile;
    k_fe_flux_combine<<<tiles, kScanTile, 0, st>>>(M, n_sys, wb);
    count_launch();
    k_fe_flux_scan<<<tiles, kScanTile, 0, st>>>(M, n_sys, wb, u_mean);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
  }
  double* w = static_cast<double*>(work);
  k_fe_spike<<<(unsigned)n_sys, kFeChunks, 0, st>>>(B, ldb, M, g_hat, w);
  count_launch();
  const int slots = fe_chunk_rows(M - 1) * kFeChunks;
  k_fe_mean2<<<(slots + 31) / 32, 256, 0, st>>>(w, n_sys, M, u_mean);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // extern "C"
