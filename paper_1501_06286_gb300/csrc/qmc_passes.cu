// qmc_passes.cu — FP32 instantiations of the pass kernel, their launcher,
// tile-shape selection, row 0 and point generation.
#include <math.h>

#include "qmc_pass_kernel.cuh"

namespace qmc {

static unsigned long long g_launches = 0;
void count_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
unsigned long long launch_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
void add_launches(long long delta) {
  __atomic_add_fetch(&g_launches, (unsigned long long)delta, __ATOMIC_RELAXED);
}

bool factor_radices(int LP, Radices* out) {
  // Greedy: radix 16 first, then 8, 4, 2 for the power of two, then the
  // odd primes the butterflies cover.
  Radices rd{};
  if (LP == 257) {  // prime factor handled by Rader's algorithm
    rd.n = 1;
    rd.r[0] = kRader257;
    *out = rd;
    return true;
  }
  int n = LP;
  auto push = [&](int r) {
    if (rd.n >= kMaxStages) return false;
    rd.r[rd.n++] = r;
    n /= r;
    return true;
  };
  while (n % 16 == 0) if (!push(16)) return false;
  if (n % 8 == 0 && !push(8)) return false;
  if (n % 4 == 0 && !push(4)) return false;
  if (n % 2 == 0 && !push(2)) return false;
  const int odd[] = {3, 5, 7, 11, 13, 17};
  for (int q : odd)
    while (n % q == 0) if (!push(q)) return false;
  if (n != 1) return false;
  *out = rd;
  return true;
}

static int ilog2(int x) { int l = 0; while ((1 << l) < x) ++l; return l; }

int choose_tile(int LP, int T, int elem_bytes, int n_linegroups, int* logW, int* logV) {
  // W: complex columns per panel (up to 8 = 64 bytes of FP32 pairs);
  // V: line groups per tile, so that a tile holds <= 8192 FP32 (4096 FP64)
  // elements and a block of <= 1024 threads covers it at kEPT per thread.
  int W = 1;
  while (W < 8 && W < T) W <<= 1;
  const int cap = elem_bytes == 8 ? 8192 : 4096;
  int V = 1;
  while (V < 32 && (int64_t)LP * W * V * 2 <= cap && V < n_linegroups) V <<= 1;
  if ((int64_t)LP * W * V > (int64_t)kEPT * 512) return -1;
  *logW = ilog2(W);
  *logV = ilog2(V);
  return 0;
}

template <typename R, int LOAD, int STORE>
static int run(const PassArgs& a, cudaStream_t st) {
  const int items = a.LP << a.logM;
  int nt = (items + kEPT - 1) / kEPT;
  nt = ((nt + 31) / 32) * 32;
  if (nt < 32) nt = 32;
  if (nt > 512) return QMC_ERR_UNSUPPORTED;
  const bool rader = a.nst == 1 && (int)(a.rbits & 31u) == kRader257;
  const size_t smem = sizeof(cx<R>) * ((size_t)a.LP + 2 * (size_t)items +
                                       (rader ? 256 + 2 * ((size_t)1 << a.logM) : 0));
  // Opt in to the dynamic shared memory this launch needs (above the
  // 48 KB default); a refusal leaves no pending error behind.
  static KernelSetup setup;
  if (const int rc = setup_kernel(k_pass<R, LOAD, STORE>, setup, smem, nt, nullptr)) return rc;
  const int V = 1 << a.logV;
  dim3 grid((a.n_linegroups + V - 1) / V, (a.T + (1 << a.logW) - 1) >> a.logW);
  k_pass<R, LOAD, STORE><<<grid, nt, smem, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

int launch_pass_f64(const PassArgs& a, int load, int store, cudaStream_t st);

int launch_pass(const PassArgs& a, int R_is_double, int load, int store, cudaStream_t st) {
  if (R_is_double) return launch_pass_f64(a, load, store, st);
  if (load == LD_GATHER_A && store == ST_SCRATCH) return run<float, LD_GATHER_A, ST_SCRATCH>(a, st);
  if (load == LD_SCRATCH && store == ST_SCRATCH) return run<float, LD_SCRATCH, ST_SCRATCH>(a, st);
  if (load == LD_SCRATCH && store == ST_OUT) return run<float, LD_SCRATCH, ST_OUT>(a, st);
  if (load == LD_GATHER_A && store == ST_OUT) return run<float, LD_GATHER_A, ST_OUT>(a, st);
  if (load == LD_PERM_G && store == ST_SCRATCH) return run<float, LD_PERM_G, ST_SCRATCH>(a, st);
  if (load == LD_SCRATCH && store == ST_DA) return run<float, LD_SCRATCH, ST_DA>(a, st);
  if (load == LD_PERM_G && store == ST_DA) return run<float, LD_PERM_G, ST_DA>(a, st);
  if (load == LD_PSET && store == ST_SCRATCH) return run<float, LD_PSET, ST_SCRATCH>(a, st);
  if (load == LD_SCRATCH && store == ST_PSET) return run<float, LD_SCRATCH, ST_PSET>(a, st);
  if (load == LD_PSET && store == ST_PSET) return run<float, LD_PSET, ST_PSET>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

// ---------------------------------------------------------------------------
// Y materialised from Eq. (3): Y'[r][j] = z_{(e_j - r) mod L}, row r of the
// circulant order written to output row out_row(r); row 0 = φ(0).
// ---------------------------------------------------------------------------
__global__ void k_points(const double* zeta, const int* e, const int* orow, int64_t L, int s,
                         float* Y, int64_t ldy, int has_row0, float phi0, int64_t n_out, int* err) {
  const int64_t r = blockIdx.x;  // circulant row, or L for row 0
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < s; j += gridDim.y * blockDim.x) {
    if (r < L) {
      int64_t k = chk((int64_t)e[j], L, err) - r;
      if (k < 0) k += L;
      Y[chk((int64_t)orow[r], n_out, err) * ldy + j] = (float)zeta[k];
    } else if (has_row0) {
      Y[j] = phi0;
    }
  }
}

// Korobov p-set (Section 2.2): block b, circulant row r holds
// Y'_b[r][j] = z_{(j·b - r) mod L}, written to row ps_blk[b]·L + out_row(r).
__global__ void k_points_pset(const double* zeta, const int* orow, const int* blk, int64_t L, int s,
                              float* Y, int64_t ldy, int* err) {
  const int64_t br = blockIdx.x;  // b·L + r
  const int64_t b = br / L, r = br - b * L;
  const int64_t row = chk((int64_t)blk[b], L, err) * L + chk((int64_t)orow[r], L, err);
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < s; j += gridDim.y * blockDim.x) {
    int64_t k = ((int64_t)j * b) % L - r;
    if (k < 0) k += L;
    Y[row * ldy + j] = (float)zeta[k];
  }
}

int launch_generate_points(const Plan& p, float* Y, int64_t ldy, cudaStream_t st) {
  const int nt = 256;
  if (p.pset) {
    if (p.L * p.L > 0x7fffffff) return QMC_ERR_UNSUPPORTED;  // one block per output row
    int gy = (p.s + nt - 1) / nt;
    if (gy > 64) gy = 64;
    dim3 grid((unsigned)(p.L * p.L), gy);
    k_points_pset<<<grid, nt, 0, st>>>(p.d_zeta, p.d_orow, p.d_ps_blk, p.L, p.s, Y, ldy, p.d_err);
    return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
  }
  int gy = (p.s + nt - 1) / nt;
  if (gy > 64) gy = 64;
  dim3 grid((unsigned)(p.L + (p.has_row0 ? 1 : 0)), gy);
  k_points<<<grid, nt, 0, st>>>(p.d_zeta, p.d_e, p.d_orow, p.L, p.s, Y, ldy, p.has_row0,
                                (float)p.phi0, p.out_rows, p.d_err);
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // namespace qmc
