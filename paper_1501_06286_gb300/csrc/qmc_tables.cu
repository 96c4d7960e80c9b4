// qmc_tables.cu — plan-time kernels: powers and discrete logs of the
// primitive element, the exponents e_j, the position -> j lists of the
// scatter-add, the output-row permutation, the generator sequence z_k and
// its FP64 spectrum (Section 2.1; Remark 1 for F_2).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "qmc_internal.h"

namespace qmc {

// ---------------------------------------------------------------------------
// Prime field: pow[k] = g^k mod N (k < L = N-1), by square-and-multiply in
// 64-bit integers (N < 2^31 so products fit).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mulmod(uint64_t a, uint64_t b, uint64_t N) { return (a * b) % N; }

__global__ void k_pow_prime(int64_t L, uint64_t N, uint64_t g, int* pw) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = 1, b = g % N;
    uint64_t e = (uint64_t)k;
    while (e) {
      if (e & 1) r = mulmod(r, b, N);
      b = mulmod(b, b, N);
      e >>= 1;
    }
    pw[k] = (int)r;
  }
}

// ---------------------------------------------------------------------------
// F_2[x]/(P): pow[k] = x^k mod P as an m-bit integer (bit i = coeff of x^i).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t clmul32(uint32_t a, uint32_t b) {
  uint64_t r = 0;
  for (int i = 0; i < 32; ++i)
    if ((b >> i) & 1u) r ^= (uint64_t)a << i;
  return r;
}
__device__ __forceinline__ uint32_t polymod(uint64_t a, uint64_t P, int m) {
  for (int d = 2 * m - 2; d >= m; --d)
    if ((a >> d) & 1ull) a ^= P << (d - m);
  return (uint32_t)a;
}

__global__ void k_pow_f2(int64_t L, uint64_t P, int m, int* pw) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint32_t r = 1, b = polymod(2u, P, m);
    uint64_t e = (uint64_t)k;
    while (e) {
      if (e & 1) r = polymod(clmul32(r, b), P, m);
      b = polymod(clmul32(b, b), P, m);
      e >>= 1;
    }
    pw[k] = (int)r;
  }
}

// ---------------------------------------------------------------------------
// F_b[x]/(P), b prime: pow[k] = x^k mod P as the base-b integer Σ c_i b^i.
// Each thread takes a run of kFbRun consecutive k: x^{k0} by
// square-and-multiply on digit vectors, then one multiplication by x per
// step (shift the digits up, subtract c·P for the carried-out digit c).
// ---------------------------------------------------------------------------
constexpr int kFbMaxM = 31;
constexpr int kFbRun = 64;

__device__ void fb_mul(const uint8_t* a, const uint8_t* c, const uint8_t* P, int b, int m, uint8_t* out) {
  int prod[2 * kFbMaxM];
  for (int i = 0; i < 2 * m; ++i) prod[i] = 0;
  for (int i = 0; i < m; ++i)
    if (a[i])
      for (int j = 0; j < m; ++j) prod[i + j] = (prod[i + j] + a[i] * c[j]) % b;
  for (int d = 2 * m - 2; d >= m; --d) {
    const int q = prod[d];
    if (!q) continue;
    for (int i = 0; i <= m; ++i) prod[d - m + i] = (prod[d - m + i] + (b - q) * P[i]) % b;
  }
  for (int i = 0; i < m; ++i) out[i] = (uint8_t)prod[i];
}

__global__ void k_pow_fb(int64_t L, uint64_t Penc, int b, int m, int* pw) {
  uint8_t P[kFbMaxM + 1];
  {
    uint64_t v = Penc;
    for (int i = 0; i <= m; ++i) { P[i] = (uint8_t)(v % (uint64_t)b); v /= (uint64_t)b; }
  }
  const int64_t nruns = (L + kFbRun - 1) / kFbRun;
  for (int64_t run = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; run < nruns;
       run += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k0 = run * kFbRun;
    uint8_t r[kFbMaxM], x[kFbMaxM], t[kFbMaxM];
    for (int i = 0; i < m; ++i) { r[i] = 0; x[i] = 0; }
    r[0] = 1;
    if (m == 1) x[0] = (uint8_t)((b - P[0]) % b);
    else x[1] = 1;
    for (uint64_t e = (uint64_t)k0; e; e >>= 1) {
      if (e & 1) {
        fb_mul(r, x, P, b, m, t);
        for (int i = 0; i < m; ++i) r[i] = t[i];
      }
      fb_mul(x, x, P, b, m, t);
      for (int i = 0; i < m; ++i) x[i] = t[i];
    }
    const int64_t k1 = k0 + kFbRun < L ? k0 + kFbRun : L;
    for (int64_t k = k0; k < k1; ++k) {
      int64_t v = 0;
      for (int i = m - 1; i >= 0; --i) v = v * b + r[i];
      pw[k] = (int)v;
      const int c = r[m - 1];  // x·r: the digit carried to x^m is reduced by P
      for (int i = m - 1; i > 0; --i) r[i] = (uint8_t)((r[i - 1] + (b - c) * P[i]) % b);
      r[0] = (uint8_t)(((b - c) * P[0]) % b);
    }
  }
}

// log[pow[k]] = k; the caller pre-fills log with -1.
__global__ void k_log(int64_t L, const int* pw, int* lg) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L;
       k += (int64_t)gridDim.x * blockDim.x)
    lg[pw[k]] = (int)k;
}

// Counts values 1..n-1 that no power reached (0 iff g, resp. x, is primitive).
__global__ void k_check_log(int64_t n, const int* lg, int* missing) {
  int local = 0;
  for (int64_t v = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    local += lg[v] < 0;
  if (local) atomicAdd(missing, local);
}

// e_j = log z_j (prime), log q_j (F_2), or e_j given.
__global__ void k_exponents(const int64_t* gen, int s, int is_exp, int kind, int64_t N, int64_t L,
                            const int* lg, int* e, int* err) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  const int64_t gv = gen[j];
  int ej = 0;
  bool ok = true;
  if (is_exp) {
    ok = gv >= 0 && gv < L;
    ej = ok ? (int)gv : 0;
  } else if (kind == QMC_LATTICE_PRIME) {
    int64_t v = gv % N;
    if (v < 0) v += N;
    ok = v != 0;
    ej = ok ? lg[v] : 0;
  } else {
    ok = gv > 0 && gv < N;
    ej = ok ? lg[gv] : 0;
  }
  if (!ok || ej < 0) {
    atomicOr(err, kErrGenerator);
    ej = 0;
  }
  e[j] = ej;
}

__global__ void k_count(const int* e, int s, int* cnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < s) atomicAdd(cnt + e[j], 1);
}

// Exclusive scan of cnt[0..L) into row_ptr[0..L], one block; also counts
// the distinct positions.
__global__ void k_scan(const int* cnt, int64_t L, int* row_ptr, int* n_distinct) {
  __shared__ int part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t chunk = (L + nt - 1) / nt;
  const int64_t b = tid * chunk, e = b + chunk < L ? b + chunk : L;
  int sum = 0, nd = 0;
  for (int64_t i = b; i < e; ++i) { sum += cnt[i]; nd += cnt[i] > 0; }
  part[tid] = sum;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    const int v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int run = part[tid] - sum;  // exclusive prefix of this chunk
  for (int64_t i = b; i < e; ++i) { row_ptr[i] = run; run += cnt[i]; }
  if (tid == nt - 1) row_ptr[L] = part[nt - 1];
  if (nd) atomicAdd(n_distinct, nd);
}

__global__ void k_fill(const int* e, int s, int* cursor, int* jlist) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < s) jlist[atomicAdd(cursor + e[j], 1)] = j;
}

// Sort each colliding position's j list so that the scatter-add sums in a
// fixed order (deterministic results).
__global__ void k_sort_segments(int64_t L, const int* row_ptr, int* jlist) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < L;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int b = row_ptr[u], e = row_ptr[u + 1];
    for (int i = b + 1; i < e; ++i) {
      const int x = jlist[i];
      int k = i - 1;
      while (k >= b && jlist[k] > x) { jlist[k + 1] = jlist[k]; --k; }
      jlist[k + 1] = x;
    }
  }
}

// Non-empty positions u = n1*NB + b of first-pass line b, in increasing n1.
__global__ void k_bucket_count(int NB, int L1, const int* row_ptr, int* bcnt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= NB) return;
  int c = 0;
  for (int n1 = 0; n1 < L1; ++n1) {
    const int64_t u = (int64_t)n1 * NB + b;
    c += row_ptr[u + 1] > row_ptr[u];
  }
  bcnt[b] = c;
}

__global__ void k_bucket_fill(int NB, int L1, const int* row_ptr, const int* bucket_ptr, int* blist) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= NB) return;
  int o = bucket_ptr[b];
  for (int n1 = 0; n1 < L1; ++n1) {
    const int64_t u = (int64_t)n1 * NB + b;
    if (row_ptr[u + 1] > row_ptr[u]) blist[o++] = (int)u;
  }
}

// Entries (point index, j) of first-pass line b: all j whose e_j = n1*NB + b,
// in increasing n1 and, within a position, increasing j.  Count pass first
// (largest count into *emax), then the padded fill.
__global__ void k_gather_count(int NB, const int* bucket_ptr, const int* blist, const int* row_ptr,
                               int* emax) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= NB) return;
  int c = 0;
  for (int q = bucket_ptr[b]; q < bucket_ptr[b + 1]; ++q) {
    const int u = blist[q];
    c += row_ptr[u + 1] - row_ptr[u];
  }
  atomicMax(emax, c);
}

__global__ void k_gather_fill(int NB, int em, const int* bucket_ptr, const int* blist,
                              const int* row_ptr, const int* jlist, int* gp_i, int* gp_j) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= NB) return;
  int o = b * em;
  for (int q = bucket_ptr[b]; q < bucket_ptr[b + 1]; ++q) {
    const int u = blist[q];
    for (int k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
      gp_i[o] = u / NB;   // u = n1*NB + b
      gp_j[o] = jlist[k];
      ++o;
    }
  }
  for (; o < (b + 1) * em; ++o) { gp_i[o] = -1; gp_j[o] = 0; }
}

// Output row of circulant row r.  Section 2.1: reordered point n = r + 1
// has conventional index g^{-r} mod N = pow[(L - r) mod L]; for F_2 the
// point with n(x) = x^{-r} mod P, i.e. the integer pow[(L - r) mod L].
__global__ void k_orow(int64_t L, const int* pw, int order, int has_row0, int* orow) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (order == QMC_ORDER_CIRCULANT) {
      orow[r] = (int)(r + has_row0);
    } else {
      const int64_t k = r == 0 ? 0 : L - r;
      orow[r] = pw[k] - (has_row0 ? 0 : 1);
    }
  }
}

__device__ __forceinline__ double apply_map(double x, int map) {
  switch (map) {
    case QMC_MAP_IDENTITY: return x;
    case QMC_MAP_CENTRED: return x - 0.5;
    case QMC_MAP_TENT: return 1.0 - fabs(2.0 * x - 1.0);
    case QMC_MAP_PHI_INV: return normcdfinv(x);
    default: return 0.0;
  }
}

// z_k = φ(x_k).  Prime: x_k = (g^k mod N)/N.  F_2 (F_b): x_k = v_m(x^k mod P / P)
// whose Laurent digits are the top bits of x^{k}, x^{k+1}, ..., x^{k+m-1}
// mod P (multiplying by x shifts the digit string by one place).
__device__ __forceinline__ double shift_mod1(double x, double delta) {
  const double y = x + delta;  // {x + Δ} for x, Δ in [0, 1)
  return y >= 1.0 ? y - 1.0 : y;
}

__global__ void k_zeta(int64_t L, const int* pw, int kind, int64_t N, int m, int base, int map, double shift,
                       double* zeta) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L;
       k += (int64_t)gridDim.x * blockDim.x) {
    double x;
    if (kind == QMC_LATTICE_PRIME) {
      x = (double)pw[k] / (double)N;
    } else if (kind == QMC_LATTICE_FB) {
      // digit u_r of x^k/P is the top coefficient (of x^{m-1}) of
      // x^{k+r-1} mod P, the same window as for F_2 in base b
      const int64_t top = N / base;
      int64_t num = 0;
      int64_t idx = k;
      for (int i = 0; i < m; ++i) {
        num = num * base + (int64_t)pw[idx] / top;
        if (++idx == L) idx = 0;
      }
      x = (double)num / (double)N;
    } else {
      uint64_t num = 0;
      int64_t idx = k;
      for (int i = 0; i < m; ++i) {
        num = (num << 1) | (((uint32_t)pw[idx] >> (m - 1)) & 1u);
        if (++idx == L) idx = 0;
      }
      x = (double)num / (double)N;
    }
    zeta[k] = apply_map(shift_mod1(x, shift), map);
  }
}

__global__ void k_map_value(int map, double x, double* out) { *out = apply_map(x, map); }

// tw[k] = exp(+2 pi i k / L) from FP64 sincospi, stored in FP64 and FP32.
__global__ void k_twiddle(int64_t L, cx<double>* tw64, cx<float>* tw32) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L;
       k += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi((double)(2 * k) / (double)L, &s, &c);
    tw64[k] = mk<double>(c, s);
    tw32[k] = mk<float>((float)c, (float)s);
  }
}

// Rader tables for p = 257 with primitive root 3 (3 * 86 = 258 = 1 mod 257):
// tw256, what_fwd, what_inv in FP64 and FP32, and the two permutations.
__global__ void k_rader_tables(cx<double>* t64, cx<float>* t32, int16_t* perm) {
  const int k = threadIdx.x;  // one block of 256 threads
  __shared__ int pout_s[256];
  int pa = 1, pb = 1;
  for (int i = 0; i < k; ++i) { pa = (pa * 3) % 257; pb = (pb * 86) % 257; }
  perm[k] = (int16_t)pa;
  perm[256 + k] = (int16_t)pb;
  pout_s[k] = pb;
  __syncthreads();
  double s, c;
  sincospi((double)(2 * k) / 256.0, &s, &c);
  t64[k] = mk<double>(c, s);
  for (int d = 0; d < 2; ++d) {
    const double dir = d == 0 ? -1.0 : 1.0;
    double re = 0.0, im = 0.0;
    for (int m = 0; m < 256; ++m) {
      double ws, wc, es, ec;
      sincospi(dir * (double)(2 * pout_s[m]) / 257.0, &ws, &wc);   // w_m
      sincospi(-(double)(2 * ((m * k) & 255)) / 256.0, &es, &ec);  // e^{-2 pi i m k/256}
      re += wc * ec - ws * es;
      im += wc * es + ws * ec;
    }
    t64[256 * (1 + d) + k] = mk<double>(re / 256.0, im / 256.0);
  }
  __syncthreads();
  for (int i = k; i < 768; i += 256) t32[i] = mk<float>((float)t64[i].re, (float)t64[i].im);
}

// H = conj(DFT(z)) / L in FP64, rounded once to FP32.
__global__ void k_spec_final(int64_t L, const cx<double>* X, cx<double>* H64, cx<float>* H32) {
  const double inv = 1.0 / (double)L;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L;
       k += (int64_t)gridDim.x * blockDim.x) {
    const cx<double> h = mk<double>(X[k].re * inv, -X[k].im * inv);
    H64[k] = h;
    H32[k] = mk<float>((float)h.re, (float)h.im);
  }
}

// Entry list of the sparse first pass (second pass of length L2 = P^2,
// P = 16 or 32): the rows of A with their positions e = n1·L2 + n2, grouped
// by n2 mod P (the spectral pass's thread t owns the points n2 ≡ t), each
// group sorted by (n2, j).
static int build_sparse_entries(Plan& p) {
  const int P = p.L2 == 256 ? 16 : 32;
  const int L2 = p.L2;
  std::vector<int> idx(p.s), pos(p.s), row(p.s), gptr(P + 1, 0);
  for (int j = 0; j < p.s; ++j) idx[j] = j;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) {
    const int ux = p.e_host[x] % L2, uy = p.e_host[y] % L2;
    if (ux % P != uy % P) return ux % P < uy % P;
    if (ux != uy) return ux < uy;
    return x < y;
  });
  for (int q = 0; q < p.s; ++q) {
    const int j = idx[q], u = p.e_host[j];
    pos[q] = ((u / L2) << 16) | (u % L2);
    row[q] = j;
    ++gptr[(u % L2) % P + 1];
  }
  for (int g = 0; g < P; ++g) gptr[g + 1] += gptr[g];
  if (cudaMalloc(&p.d_sp_pos, sizeof(int) * p.s) != cudaSuccess ||
      cudaMalloc(&p.d_sp_row, sizeof(int) * p.s) != cudaSuccess ||
      cudaMalloc(&p.d_sp_gptr, sizeof(int) * (P + 1)) != cudaSuccess ||
      cudaMemcpy(p.d_sp_pos, pos.data(), sizeof(int) * p.s, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p.d_sp_row, row.data(), sizeof(int) * p.s, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p.d_sp_gptr, gptr.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return QMC_ERR_CUDA;
  }
  p.sp_P = P;
  return QMC_OK;
}

#define QMC_CHECK(x)                                  \
  do {                                                \
    if ((x) != cudaSuccess) { rc = QMC_ERR_CUDA; goto done; } \
  } while (0)

static int grid_for(int64_t n, int nt) {
  int64_t g = (n + nt - 1) / nt;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

int build_tables(Plan& p, const int64_t* gen_host, int gen_is_exponent, cudaStream_t st) {
  int rc = QMC_OK;
  const int64_t L = p.L;
  const int nt = 256;
  int64_t* d_gen = nullptr;
  int *d_cnt = nullptr, *d_cursor = nullptr, *d_counters = nullptr;
  cx<double>* d_tw64 = nullptr;
  cx<double>* d_x64 = nullptr;
  int host_counters[2] = {0, 0};
  int host_err = 0;

  p.log_size = p.N;
  QMC_CHECK(cudaMalloc(&p.d_pow, sizeof(int) * L));
  QMC_CHECK(cudaMalloc(&p.d_log, sizeof(int) * p.log_size));
  QMC_CHECK(cudaMalloc(&p.d_e, sizeof(int) * p.s));
  QMC_CHECK(cudaMalloc(&p.d_row_ptr, sizeof(int) * (L + 1)));
  QMC_CHECK(cudaMalloc(&p.d_jlist, sizeof(int) * p.s));
  QMC_CHECK(cudaMalloc(&p.d_bucket_ptr, sizeof(int) * (p.L2 + 1)));
  QMC_CHECK(cudaMalloc(&p.d_blist, sizeof(int) * p.s));
  QMC_CHECK(cudaMalloc(&p.d_abar, sizeof(double) * p.s));
  QMC_CHECK(cudaMalloc(&p.d_orow, sizeof(int) * L));
  QMC_CHECK(cudaMalloc(&p.d_zeta, sizeof(double) * L));
  QMC_CHECK(cudaMalloc(&p.d_H, sizeof(cx<float>) * L));
  QMC_CHECK(cudaMalloc(&p.d_H64, sizeof(cx<double>) * L));
  QMC_CHECK(cudaMalloc(&p.d_tw, sizeof(cx<float>) * L));
  QMC_CHECK(cudaMalloc(&p.d_err, sizeof(int)));
  QMC_CHECK(cudaMalloc(&d_gen, sizeof(int64_t) * p.s));
  QMC_CHECK(cudaMalloc(&d_cnt, sizeof(int) * L));
  QMC_CHECK(cudaMalloc(&d_cursor, sizeof(int) * (L + 1)));
  QMC_CHECK(cudaMalloc(&d_counters, sizeof(int) * 3));
  QMC_CHECK(cudaMalloc(&d_tw64, sizeof(cx<double>) * L));
  QMC_CHECK(cudaMalloc(&d_x64, sizeof(cx<double>) * L));
  QMC_CHECK(cudaMemsetAsync(p.d_err, 0, sizeof(int), st));
  QMC_CHECK(cudaMemsetAsync(d_counters, 0, sizeof(int) * 3, st));
  QMC_CHECK(cudaMemsetAsync(p.d_log, 0xff, sizeof(int) * p.log_size, st));
  QMC_CHECK(cudaMemsetAsync(d_cnt, 0, sizeof(int) * L, st));
  QMC_CHECK(cudaMemcpyAsync(d_gen, gen_host, sizeof(int64_t) * p.s, cudaMemcpyHostToDevice, st));

  if (p.kind == QMC_LATTICE_PRIME)
    k_pow_prime<<<grid_for(L, nt), nt, 0, st>>>(L, (uint64_t)p.N, (uint64_t)p.g, p.d_pow);
  else if (p.kind == QMC_LATTICE_FB)
    k_pow_fb<<<grid_for((L + kFbRun - 1) / kFbRun, nt), nt, 0, st>>>(L, p.P, p.base, p.m, p.d_pow);
  else
    k_pow_f2<<<grid_for(L, nt), nt, 0, st>>>(L, p.P, p.m, p.d_pow);
  k_log<<<grid_for(L, nt), nt, 0, st>>>(L, p.d_pow, p.d_log);
  k_check_log<<<grid_for(p.log_size, nt), nt, 0, st>>>(p.log_size, p.d_log, d_counters + 0);
  k_exponents<<<(p.s + nt - 1) / nt, nt, 0, st>>>(d_gen, p.s, gen_is_exponent, p.kind, p.N, L,
                                                  p.d_log, p.d_e, p.d_err);
  k_count<<<(p.s + nt - 1) / nt, nt, 0, st>>>(p.d_e, p.s, d_cnt);
  k_scan<<<1, 1024, 0, st>>>(d_cnt, L, p.d_row_ptr, d_counters + 1);
  QMC_CHECK(cudaMemcpyAsync(d_cursor, p.d_row_ptr, sizeof(int) * (L + 1), cudaMemcpyDeviceToDevice, st));
  k_fill<<<(p.s + nt - 1) / nt, nt, 0, st>>>(p.d_e, p.s, d_cursor, p.d_jlist);
  k_sort_segments<<<grid_for(L, nt), nt, 0, st>>>(L, p.d_row_ptr, p.d_jlist);
  // first-pass line buckets (d_cnt is reused for the per-line counts)
  k_bucket_count<<<(p.L2 + nt - 1) / nt, nt, 0, st>>>(p.L2, p.L1, p.d_row_ptr, d_cnt);
  k_scan<<<1, 1024, 0, st>>>(d_cnt, p.L2, p.d_bucket_ptr, d_counters + 2);
  k_bucket_fill<<<(p.L2 + nt - 1) / nt, nt, 0, st>>>(p.L2, p.L1, p.d_row_ptr, p.d_bucket_ptr, p.d_blist);
  k_orow<<<grid_for(L, nt), nt, 0, st>>>(L, p.d_pow, p.order, p.has_row0, p.d_orow);
  k_zeta<<<grid_for(L, nt), nt, 0, st>>>(L, p.d_pow, p.kind, p.N, p.m, p.base, p.map, p.shift, p.d_zeta);
  k_twiddle<<<grid_for(L, nt), nt, 0, st>>>(L, d_tw64, p.d_tw);
  if (p.L1 == 257 || p.L2 == 257) {
    QMC_CHECK(cudaMalloc(&p.d_rader32, sizeof(cx<float>) * 768));
    QMC_CHECK(cudaMalloc(&p.d_rader64, sizeof(cx<double>) * 768));
    QMC_CHECK(cudaMalloc(&p.d_rader_perm, sizeof(int16_t) * 512));
    k_rader_tables<<<1, 256, 0, st>>>(p.d_rader64, p.d_rader32, p.d_rader_perm);
  }
  QMC_CHECK(cudaGetLastError());

  {
    // Spectrum of z in FP64 through the same pass kernel (one column).
    PassArgs a{};
    a.L = (int)L;
    a.T = 1;
    a.t = 1;
    a.scratch = d_x64;
    a.twL = d_tw64;
    a.zeta = p.d_zeta;
    a.err = p.d_err;
    a.rader = p.d_rader64;
    a.rader_perm = p.d_rader_perm;
    a.fwd = 1;
    if (p.L2 == 1) {
      a.LP = p.L1; a.nst = p.rad1.n; a.rbits = p.rad1.packed(); a.point_stride = 1; a.line_stride = 1; a.n_linegroups = 1;
      if (choose_tile(a.LP, 1, 16, 1, &a.logW, &a.logV)) { rc = QMC_ERR_UNSUPPORTED; goto done; }
      a.logM = a.logW + a.logV;
      rc = launch_pass(a, 1, LD_DENSE64, ST_SCRATCH, st);
      if (rc) goto done;
    } else {
      a.LP = p.L1; a.nst = p.rad1.n; a.rbits = p.rad1.packed(); a.point_stride = p.L2; a.line_stride = 1;
      a.n_linegroups = p.L2; a.twiddle = -1;
      if (choose_tile(a.LP, 1, 16, a.n_linegroups, &a.logW, &a.logV)) { rc = QMC_ERR_UNSUPPORTED; goto done; }
      a.logM = a.logW + a.logV;
      rc = launch_pass(a, 1, LD_DENSE64, ST_SCRATCH, st);
      if (rc) goto done;
      PassArgs b = a;
      b.LP = p.L2; b.nst = p.rad2.n; b.rbits = p.rad2.packed(); b.point_stride = 1; b.line_stride = p.L2;
      b.n_linegroups = p.L1; b.twiddle = 0;
      if (choose_tile(b.LP, 1, 16, b.n_linegroups, &b.logW, &b.logV)) { rc = QMC_ERR_UNSUPPORTED; goto done; }
      b.logM = b.logW + b.logV;
      rc = launch_pass(b, 1, LD_SCRATCH, ST_SCRATCH, st);
      if (rc) goto done;
    }
    k_spec_final<<<grid_for(L, nt), nt, 0, st>>>(L, d_x64, p.d_H64, p.d_H);
    QMC_CHECK(cudaGetLastError());
  }

  QMC_CHECK(cudaMemcpyAsync(host_counters, d_counters, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  QMC_CHECK(cudaMemcpyAsync(&host_err, p.d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  QMC_CHECK(cudaStreamSynchronize(st));
  if (host_counters[0] != 0) { rc = QMC_ERR_NOT_PRIMITIVE; goto done; }
  if (host_err & kErrGenerator) { rc = QMC_ERR_GENERATOR; goto done; }
  if (p.L2 > 1) {
    // padded first-pass gather table, when every line has few entries
    int em = 0;
    QMC_CHECK(cudaMemsetAsync(d_counters, 0, sizeof(int), st));
    k_gather_count<<<(p.L2 + nt - 1) / nt, nt, 0, st>>>(p.L2, p.d_bucket_ptr, p.d_blist, p.d_row_ptr,
                                                        d_counters);
    QMC_CHECK(cudaMemcpyAsync(&em, d_counters, sizeof(int), cudaMemcpyDeviceToHost, st));
    QMC_CHECK(cudaStreamSynchronize(st));
    if (em >= 1 && em <= kGatherMax) {
      QMC_CHECK(cudaMalloc(&p.d_gp_i, sizeof(int) * (size_t)p.L2 * em));
      QMC_CHECK(cudaMalloc(&p.d_gp_j, sizeof(int) * (size_t)p.L2 * em));
      k_gather_fill<<<(p.L2 + nt - 1) / nt, nt, 0, st>>>(p.L2, em, p.d_bucket_ptr, p.d_blist,
                                                         p.d_row_ptr, p.d_jlist, p.d_gp_i, p.d_gp_j);
      QMC_CHECK(cudaGetLastError());
      p.gp_em = em;
      // lines by entry count: term-by-term lines first, then the others
      std::vector<int> gi((size_t)p.L2 * em), order;
      QMC_CHECK(cudaMemcpy(gi.data(), p.d_gp_i, sizeof(int) * gi.size(), cudaMemcpyDeviceToHost));
      std::vector<int> cnt((size_t)p.L2), single, fft;
      for (int b = 0; b < p.L2; ++b) {
        int n = 0;
        while (n < em && gi[(size_t)b * em + n] >= 0) ++n;
        cnt[(size_t)b] = n;
      }
      // neighbouring lines 2λ, 2λ+1 that both take the term-by-term sums
      // run as one tile (their points sit in neighbouring rows)
      for (int b = 0; b < p.L2; ++b) {
        const bool dir = cnt[(size_t)b] <= kDirectEntries;
        if (dir && (b & 1) == 0 && b + 1 < p.L2 && cnt[(size_t)b + 1] <= kDirectEntries) {
          order.push_back(b);
          ++b;
          continue;
        }
        (dir ? single : fft).push_back(b);
      }
      p.n_pair = (int)order.size();
      p.n_direct = (int)single.size();
      p.n_fft = (int)fft.size();
      order.insert(order.end(), single.begin(), single.end());
      order.insert(order.end(), fft.begin(), fft.end());
      QMC_CHECK(cudaMalloc(&p.d_lines, sizeof(int) * (size_t)p.L2));
      QMC_CHECK(cudaMemcpy(p.d_lines, order.data(), sizeof(int) * (size_t)p.L2, cudaMemcpyHostToDevice));
    }
  }
  p.n_distinct = host_counters[1];
  p.e_host.resize(p.s);
  QMC_CHECK(cudaMemcpy(p.e_host.data(), p.d_e, sizeof(int) * p.s, cudaMemcpyDeviceToHost));
  if (p.L2 == 256 || p.L2 == 1024) rc = build_sparse_entries(p);

done:
  cudaFree(d_gen);
  cudaFree(d_cnt);
  cudaFree(d_cursor);
  cudaFree(d_counters);
  cudaFree(d_tw64);
  cudaFree(d_x64);
  return rc;
}

int map_value(int map, double x, double* out, cudaStream_t st) {
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double)) != cudaSuccess) return QMC_ERR_ALLOC;
  k_map_value<<<1, 1, 0, st>>>(map, x, d);
  int rc = cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
  if (rc == QMC_OK && (cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess))
    rc = QMC_ERR_CUDA;
  cudaFree(d);
  return rc;
}

}  // namespace qmc
