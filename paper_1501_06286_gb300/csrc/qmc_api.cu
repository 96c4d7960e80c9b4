// qmc_api.cu — the C ABI of libqmcfft (declared in include/qmc.h): plan
// validation and construction, product orchestration, adjoint, point
// generation and batching.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <initializer_list>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qmc_internal.h"
#include "qmc_debug.h"

using namespace qmc;

namespace {

// ---------------- host integer helpers (validation only) -------------------
bool is_prime_u64(int64_t n) {
  if (n < 2) return false;
  if (n % 2 == 0) return n == 2;
  for (int64_t d = 3; d * d <= n; d += 2)
    if (n % d == 0) return false;
  return true;
}

std::vector<int64_t> prime_factors(int64_t n) {
  std::vector<int64_t> f;
  for (int64_t d = 2; d * d <= n; ++d) {
    if (n % d == 0) {
      f.push_back(d);
      while (n % d == 0) n /= d;
    }
  }
  if (n > 1) f.push_back(n);
  return f;
}

uint64_t powmod(uint64_t b, uint64_t e, uint64_t N) {
  uint64_t r = 1 % N;
  b %= N;
  while (e) {
    if (e & 1) r = (r * b) % N;
    b = (b * b) % N;
    e >>= 1;
  }
  return r;
}

bool is_primitive_root(int64_t g, int64_t N) {
  if (g < 1 || g >= N) return false;
  if (N == 2) return g == 1;
  const int64_t L = N - 1;
  for (int64_t p : prime_factors(L))
    if (powmod((uint64_t)g, (uint64_t)(L / p), (uint64_t)N) == 1) return false;
  return true;
}

uint64_t f2_mulmod(uint64_t a, uint64_t b, uint64_t P, int m) {
  uint64_t r = 0;
  for (int i = 0; i < m; ++i)
    if ((b >> i) & 1) r ^= a << i;
  for (int d = 2 * m - 2; d >= m; --d)
    if ((r >> d) & 1) r ^= P << (d - m);
  return r;
}

uint64_t f2_xpow(uint64_t e, uint64_t P, int m) {
  uint64_t r = 1, b = 2;
  if (m == 1) b = 2 ^ P;
  while (e) {
    if (e & 1) r = f2_mulmod(r, b, P, m);
    b = f2_mulmod(b, b, P, m);
    e >>= 1;
  }
  return r;
}

bool f2_is_primitive(uint64_t P, int m) {
  if (!(P & 1) || ((P >> m) != 1)) return false;
  const int64_t L = (int64_t(1) << m) - 1;
  if (f2_xpow((uint64_t)L, P, m) != 1) return false;
  for (int64_t p : prime_factors(L))
    if (p != L && f2_xpow((uint64_t)(L / p), P, m) == 1) return false;
  return true;
}

// F_b[x]/(P) for a prime b: polynomials of degree < m as digit vectors
// (coefficient of x^i at index i), P monic of degree m given by its digits.
std::vector<int> fb_digits(uint64_t v, int b, int n) {
  std::vector<int> d((size_t)n);
  for (int i = 0; i < n; ++i) { d[(size_t)i] = (int)(v % (uint64_t)b); v /= (uint64_t)b; }
  return d;
}

std::vector<int> fb_mulmod(const std::vector<int>& a, const std::vector<int>& c, const std::vector<int>& P,
                           int b, int m) {
  std::vector<int64_t> prod((size_t)(2 * m), 0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) prod[(size_t)(i + j)] += (int64_t)a[(size_t)i] * c[(size_t)j];
  for (auto& v : prod) v %= b;
  for (int d = 2 * m - 2; d >= m; --d) {
    const int64_t q = prod[(size_t)d] % b;
    if (!q) continue;
    for (int i = 0; i <= m; ++i) prod[(size_t)(d - m + i)] = ((prod[(size_t)(d - m + i)] - q * P[(size_t)i]) % b + b) % b;
  }
  std::vector<int> r((size_t)m);
  for (int i = 0; i < m; ++i) r[(size_t)i] = (int)prod[(size_t)i];
  return r;
}

bool fb_is_one(const std::vector<int>& a) {
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i] != (i == 0 ? 1 : 0)) return false;
  return true;
}

std::vector<int> fb_xpow(uint64_t e, const std::vector<int>& P, int b, int m) {
  std::vector<int> r((size_t)m, 0), x((size_t)m, 0);
  r[0] = 1;
  if (m == 1) x[0] = (b - P[0]) % b;  // x ≡ -p_0 mod (x + p_0)
  else x[1] = 1;
  while (e) {
    if (e & 1) r = fb_mulmod(r, x, P, b, m);
    x = fb_mulmod(x, x, P, b, m);
    e >>= 1;
  }
  return r;
}

// P (base-b encoding, leading digit 1 at b^m) is primitive iff x has order
// b^m - 1 modulo P.
bool fb_is_primitive(uint64_t Penc, int b, int m, int64_t L) {
  const std::vector<int> P = fb_digits(Penc, b, m + 1);
  if (P[(size_t)m] != 1 || P[0] == 0) return false;
  uint64_t top = Penc;
  for (int i = 0; i < m; ++i) top /= (uint64_t)b;
  if (top != 1) return false;
  if (!fb_is_one(fb_xpow((uint64_t)L, P, b, m))) return false;
  for (int64_t q : prime_factors(L))
    if (q != L && fb_is_one(fb_xpow((uint64_t)(L / q), P, b, m))) return false;
  return true;
}

double phi_at_zero(int map) {
  switch (map) {
    case QMC_MAP_IDENTITY: return 0.0;
    case QMC_MAP_CENTRED: return -0.5;
    case QMC_MAP_TENT: return 0.0;
    case QMC_MAP_PHI_INV: return -INFINITY;
  }
  return NAN;
}

// Korobov p-set (Section 2.2): right-hand side block b = 0..L-1 uses the
// exponents e_{b,j} = j·b mod L (j = 0..s-1).  Position u receives the j
// with j·b ≡ u (mod L): with d = gcd(b, L) there are none unless d | u,
// and then j ≡ (u/d)·(b/d)^{-1} (mod L/d).  Stores d, (b/d)^{-1} mod (L/d)
// and the block's first output row / L: γ - 1 with γ = g^b in conventional
// order, b in circulant order.
int64_t gcd64(int64_t a, int64_t b) {
  while (b) { const int64_t r = a % b; a = b; b = r; }
  return a;
}

int64_t inverse_mod64(int64_t a, int64_t m) {  // a coprime to m; m >= 1
  if (m == 1) return 0;
  int64_t r0 = m, r1 = a % m, s0 = 0, s1 = 1;
  while (r1) {
    const int64_t q = r0 / r1;
    int64_t t = r0 - q * r1; r0 = r1; r1 = t;
    t = s0 - q * s1; s0 = s1; s1 = t;
  }
  return s0 < 0 ? s0 + m : s0;
}

int build_pset_tables(Plan& p, cudaStream_t st) {
  const int64_t L = p.L;
  std::vector<int> hd((size_t)L), hinv((size_t)L), hblk((size_t)L);
  int64_t gb = 1;  // g^b mod N
  for (int64_t b = 0; b < L; ++b) {
    const int64_t d = gcd64(b, L);  // gcd(0, L) = L
    hd[(size_t)b] = (int)d;
    hinv[(size_t)b] = (int)inverse_mod64(b / d, L / d);
    hblk[(size_t)b] = (int)(p.order == QMC_ORDER_CIRCULANT ? b : gb - 1);
    gb = gb * p.g % p.N;  // N < 2^31
  }
  const size_t bytes = sizeof(int) * (size_t)L;
  if (cudaMalloc(&p.d_ps_d, bytes) != cudaSuccess || cudaMalloc(&p.d_ps_inv, bytes) != cudaSuccess ||
      cudaMalloc(&p.d_ps_blk, bytes) != cudaSuccess) {
    cudaGetLastError();
    return QMC_ERR_ALLOC;
  }
  if (cudaMemcpyAsync(p.d_ps_d, hd.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(p.d_ps_inv, hinv.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(p.d_ps_blk, hblk.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return QMC_ERR_CUDA;
  return QMC_OK;
}

// Chooses L = L1·L2 with both factors covered by the butterflies: a single
// pass when L <= 1024, else the most balanced split with factors <= 1024.
bool choose_factorisation(int64_t L, Plan& p) {
  Radices rd;
  if (L <= 1024 && factor_radices((int)L, &rd)) {
    p.L1 = (int)L; p.L2 = 1; p.rad1 = rd; p.rad2 = Radices{};
    return true;
  }
  int best1 = 0, best2 = 0;
  for (int64_t a = 2; a <= 1024 && a < L; ++a) {
    if (L % a) continue;
    const int64_t b = L / a;
    if (b > 1024 || a > b) continue;
    Radices ra, rb;
    if (!factor_radices((int)a, &ra) || !factor_radices((int)b, &rb)) continue;
    if (!best1 || std::max(a, b) < std::max<int64_t>(best1, best2)) { best1 = (int)a; best2 = (int)b; }
  }
  if (!best1) return false;
  // the longer factor (b >= a) runs as the contiguous inner pass
  p.L1 = best1; p.L2 = best2;
  factor_radices(p.L1, &p.rad1);
  factor_radices(p.L2, &p.rad2);
  return true;
}

// L = L1·L2 with the given L1 (0: the default choice); false when not a
// valid split.
bool set_factorisation(Plan& p, int64_t L1) {
  if (L1 == 0) return choose_factorisation(p.L, p);
  if (L1 < 2 || p.L % L1) return false;
  const int64_t L2 = p.L / L1;
  if (L1 > 1024 || L2 > 1024) return false;
  Radices r1, r2;
  if (!factor_radices((int)L1, &r1)) return false;
  if (L2 > 1 && !factor_radices((int)L2, &r2)) return false;
  p.L1 = (int)L1;
  p.L2 = (int)L2;
  p.rad1 = r1;
  p.rad2 = L2 > 1 ? r2 : Radices{};
  return true;
}

// Frees the tables build_tables makes (not the scratch, the statistics area
// or the profiling events) and clears their pointers.
void free_tables(Plan& p) {
  for (int** q : {&p.d_pow, &p.d_log, &p.d_e, &p.d_row_ptr, &p.d_jlist, &p.d_bucket_ptr, &p.d_blist,
                  &p.d_gp_i, &p.d_gp_j, &p.d_lines, &p.d_orow, &p.d_err, &p.d_sp_pos, &p.d_sp_row,
                  &p.d_sp_gptr}) {
    cudaFree(*q);
    *q = nullptr;
  }
  cudaFree(p.d_abar); p.d_abar = nullptr;
  cudaFree(p.d_zeta); p.d_zeta = nullptr;
  cudaFree(p.d_H); p.d_H = nullptr;
  cudaFree(p.d_H64); p.d_H64 = nullptr;
  cudaFree(p.d_tw); p.d_tw = nullptr;
  cudaFree(p.d_rader32); p.d_rader32 = nullptr;
  cudaFree(p.d_rader64); p.d_rader64 = nullptr;
  cudaFree(p.d_rader_perm); p.d_rader_perm = nullptr;
  p.gp_em = 0;
  p.n_pair = p.n_direct = p.n_fft = 0;
  p.sp_P = 0;
}

// QMC_OPT_FFT_SPLIT: a new factorisation and every table that depends on it.
int replan_split(Plan& p, int64_t L1) {
  if (p.pset) return QMC_ERR_UNSUPPORTED;
  Plan probe = {};
  probe.L = p.L;
  if (L1 != 0 && (L1 < 2 || p.L % L1 || L1 > 1024 || p.L / L1 > 1024)) return QMC_ERR_INVALID;
  if (!set_factorisation(probe, L1)) return QMC_ERR_UNSUPPORTED;
  if (probe.L1 == p.L1 && probe.L2 == p.L2) return QMC_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) return QMC_ERR_CUDA;
  const int old1 = p.L1;
  std::vector<int64_t> e(p.e_host.begin(), p.e_host.end());
  free_tables(p);
  set_factorisation(p, probe.L1 == p.L ? p.L : probe.L1);
  int rc = build_tables(p, e.data(), 1, nullptr);
  if (rc != QMC_OK) {  // back to the previous split
    free_tables(p);
    set_factorisation(p, old1);
    const int rc2 = build_tables(p, e.data(), 1, nullptr);
    if (rc2 != QMC_OK) return rc2;
  }
  return rc;
}

void free_plan(Plan* p) {
  if (!p) return;
  cudaFree(p->d_pow); cudaFree(p->d_log); cudaFree(p->d_e); cudaFree(p->d_row_ptr);
  cudaFree(p->d_jlist); cudaFree(p->d_bucket_ptr); cudaFree(p->d_blist); cudaFree(p->d_orow); cudaFree(p->d_zeta); cudaFree(p->d_H);
  cudaFree(p->d_H64); cudaFree(p->d_tw); cudaFree(p->d_err); cudaFree(p->d_scratch);
  cudaFree(p->d_stats); cudaFree(p->d_abar); cudaFree(p->d_gp_i); cudaFree(p->d_gp_j); cudaFree(p->d_lines);
  cudaFree(p->d_rader32); cudaFree(p->d_rader64); cudaFree(p->d_rader_perm);
  cudaFree(p->d_ps_d); cudaFree(p->d_ps_inv); cudaFree(p->d_ps_blk);
  cudaFree(p->d_sp_pos); cudaFree(p->d_sp_row); cudaFree(p->d_sp_gptr);
  for (auto& m : p->marks) { cudaEventDestroy(m.start); cudaEventDestroy(m.stop); }
  for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
  delete p;
}

int ensure_scratch(Plan& p, size_t bytes) {
  if (bytes <= p.scratch_bytes) return QMC_OK;
  if (p.d_scratch) { cudaFree(p.d_scratch); p.d_scratch = nullptr; p.scratch_bytes = 0; }
  if (cudaMalloc(&p.d_scratch, bytes) != cudaSuccess) { cudaGetLastError(); return QMC_ERR_ALLOC; }
  p.scratch_bytes = bytes;
  return QMC_OK;
}

int ensure_stats(Plan& p, size_t bytes) {
  if (bytes <= p.stats_bytes) return QMC_OK;
  if (p.d_stats) { cudaFree(p.d_stats); p.d_stats = nullptr; p.stats_bytes = 0; }
  if (cudaMalloc(&p.d_stats, bytes) != cudaSuccess) { cudaGetLastError(); return QMC_ERR_ALLOC; }
  p.stats_bytes = bytes;
  return QMC_OK;
}

int complex_columns(const Plan& p, int t) { return p.prec == QMC_PREC_FP32_SPLIT ? t : (t + 1) / 2; }

// AUTO takes the sparse first pass while s <= kSparseRowsPerLine·L2, about
// where it stops paying on GB300: each tile of its spectral pass reads s
// 64-byte rows of A from L2, against the first pass and the work-array
// read it saves (N = 786433, t = 1024: 20 % faster at s = 256, even at
// s = 2048; N = 65537: faster up to s ≈ 300).
constexpr int64_t kSparseRowsPerLine = 1;

// Whether a forward product of T complex columns folds its first pass into
// the spectral pass (QMC_OPT_FIRST_PASS; 8-column panels only).
bool sparse_first_pass(const Plan& p, int T) {
  if (!p.sp_P || p.pset || T < 8 || p.first_pass == QMC_FIRST_PASS_TRANSFORM) return false;
  if (p.pass_kernel != QMC_KERNEL_AUTO && p.pass_kernel != QMC_KERNEL_PIPELINED) return false;
  return p.first_pass == QMC_FIRST_PASS_SPARSE || (int64_t)p.s <= kSparseRowsPerLine * p.L2;
}

// Bytes of the L x T work array (panels of W <= 8 columns).
size_t work_bytes(const Plan& p, int T) {
  int W = 1;
  while (W < 8 && W < T) W <<= 1;
  const int64_t P = (T + W - 1) / W;
  return (size_t)P * (size_t)p.L * (size_t)W * sizeof(cx<float>);
}

// Work array, then (sparse first pass) the packed panels of A.
size_t scratch_need(const Plan& p, int t) {
  if (p.L2 == 1) return 0;  // single pass keeps everything on chip
  const int T = complex_columns(p, t);
  size_t bytes = work_bytes(p, T);
  if (sparse_first_pass(p, T)) bytes += (size_t)((T + 7) / 8) * (size_t)p.s * 8 * sizeof(cx<float>);
  return bytes;
}

bool aligned8(const void* ptr) { return ((uintptr_t)ptr & 7u) == 0; }

// Names of the stages for the NVTX ranges that bracket each launch (a
// profiler's timeline shows them; without one attached NVTX does nothing).
const char* stage_name(int stage) {
  static const char* const names[QMC_NUM_STAGES] = {
      "qmc:row0",        "qmc:fwd_scatter", "qmc:fwd_spectral", "qmc:fwd_unpermute", "qmc:fwd_fused",
      "qmc:bwd_gather",  "qmc:bwd_spectral", "qmc:bwd_scatter", "qmc:bwd_fused",     "qmc:batch",
      "qmc:row_mean",    "qmc:dense_scatter", "qmc:sparse_pack", "qmc:fwd_sparse"};
  return stage >= 0 && stage < QMC_NUM_STAGES ? names[stage] : "qmc:pass";
}

struct NvtxRange {
  explicit NvtxRange(int stage) { nvtxRangePushA(stage_name(stage)); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Runs one launch inside an NVTX range named for its stage, bracketed by
// events when the plan is profiling.
template <typename F>
int timed(Plan& p, int stage, cudaStream_t st, F&& launch) {
  NvtxRange range(stage);
  if (!p.profiling) return launch();
  // events come from the plan's pool (created once, returned by
  // qmc_plan_read_profile), so profiling adds two event records per launch
  Plan::Mark m{stage, nullptr, nullptr};
  for (cudaEvent_t* e : {&m.start, &m.stop}) {
    if (!p.event_pool.empty()) {
      *e = p.event_pool.back();
      p.event_pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      cudaGetLastError();
      return QMC_ERR_CUDA;
    }
  }
  cudaEventRecord(m.start, st);
  const int rc = launch();
  cudaEventRecord(m.stop, st);
  p.marks.push_back(m);
  return rc;
}

// One FP32 pass: the register-resident kernel for LP = 256 or 1024 unless
// the plan asks for the generic one; the generic kernel otherwise.
int pass(const Plan& p, const PassArgs& a, int load, int store, cudaStream_t st) {
  // the p-set's first and last passes run in the generic kernel
  if (load == LD_PSET || store == ST_PSET) return launch_pass(a, 0, load, store, st);
  if ((p.pass_kernel == QMC_KERNEL_AUTO || p.pass_kernel == QMC_KERNEL_PIPELINED) &&
      fast_pass_supported(a.LP)) {
    const int rc = load == LD_GATHER_A && store == ST_SCRATCH ? launch_pipe_gather(a, st)
                                                              : launch_pipe_pass(a, load, store, st);
    if (rc != QMC_ERR_UNSUPPORTED) return rc;
  }
  if (p.pass_kernel != QMC_KERNEL_GENERIC && fast_pass_supported(a.LP)) {
    const int rc = launch_fast_pass(a, load, store, st);
    if (rc != QMC_ERR_UNSUPPORTED) return rc;
  }
  if ((p.pass_kernel == QMC_KERNEL_AUTO || p.pass_kernel == QMC_KERNEL_PIPELINED) &&
      pq_pass_supported(a.LP)) {
    int rc = launch_pqpipe_pass(a, load, store, st);
    if (rc == QMC_ERR_UNSUPPORTED) rc = launch_pqpipe_spectral(a, load, store, st);
    if (rc != QMC_ERR_UNSUPPORTED) return rc;
  }
  if (p.pass_kernel != QMC_KERNEL_GENERIC && pq_pass_supported(a.LP)) {
    const int rc = launch_pq_pass(a, load, store, st);
    if (rc != QMC_ERR_UNSUPPORTED) return rc;
  }
  if (p.pass_kernel != QMC_KERNEL_GENERIC && a.LP == 257) {
    const int rc = launch_rader_spectral(a, load, store, st);
    if (rc != QMC_ERR_UNSUPPORTED) return rc;
  }
  return launch_pass(a, 0, load, store, st);
}

}  // namespace

// The FFT passes of a forward product (dir = +1) or adjoint (dir = -1):
// fills specs[0..*n) without launching anything.
int qmc::product_passes(Plan& p, int dir, PassArgs base, PassSpec* specs, int* n) {
  const int T = base.T;
  int rc;
  *n = 0;
  if ((rc = ensure_scratch(p, scratch_need(p, base.t)))) return rc;
  base.scratch = p.d_scratch;
  base.twL = p.d_tw;
  base.H = p.d_H;
  base.row_ptr = p.d_row_ptr;
  base.jlist = p.d_jlist;
  base.bucket_ptr = p.d_bucket_ptr;
  base.blist = p.d_blist;
  base.gp_i = p.d_gp_i;
  base.gp_j = p.d_gp_j;
  base.gp_em = p.gp_em;
  base.lines = p.d_lines;
  base.n_pair = p.n_pair;
  base.n_direct = p.n_direct;
  base.n_fft = p.n_fft;
  base.orow = p.d_orow;
  base.err = p.d_err;
  base.n_out = p.out_rows;
  base.s_a = p.s;
  base.L = (int)p.L;
  base.rader = p.d_rader32;
  base.rader_perm = p.d_rader_perm;
  const int first_load = p.pset ? LD_PSET : dir > 0 ? LD_GATHER_A : LD_PERM_G;
  const int last_store = p.pset ? ST_PSET : dir > 0 ? ST_OUT : ST_DA;
  const int s0 = dir > 0 ? QMC_STAGE_FWD_SCATTER : QMC_STAGE_BWD_GATHER;
  if (p.L2 == 1) {
    PassArgs a = base;
    a.LP = p.L1; a.nst = p.rad1.n; a.rbits = p.rad1.packed(); a.point_stride = 1; a.line_stride = 1; a.n_linegroups = 1;
    a.fwd = 1; a.inv = 1; a.mul = dir > 0 ? 1 : 2; a.twiddle = 0;
    if (choose_tile(a.LP, T, 8, 1, &a.logW, &a.logV)) return QMC_ERR_UNSUPPORTED;
    a.logV = 0;
    a.logM = a.logW;
    specs[(*n)++] = PassSpec{a, first_load, last_store, s0 + 3};
    return QMC_OK;
  }
  PassArgs a = base;
  a.LP = p.L1; a.nst = p.rad1.n; a.rbits = p.rad1.packed(); a.point_stride = p.L2; a.line_stride = 1; a.n_linegroups = p.L2;
  a.fwd = 1; a.inv = 0; a.mul = 0; a.twiddle = -1;
  if (choose_tile(a.LP, T, 8, a.n_linegroups, &a.logW, &a.logV)) return QMC_ERR_UNSUPPORTED;
  a.logM = a.logW + a.logV;

  PassArgs b = base;
  b.LP = p.L2; b.nst = p.rad2.n; b.rbits = p.rad2.packed(); b.point_stride = 1; b.line_stride = p.L2; b.n_linegroups = p.L1;
  b.fwd = 1; b.inv = 1; b.mul = dir > 0 ? 1 : 2; b.twiddle = +1;
  if (choose_tile(b.LP, T, 8, b.n_linegroups, &b.logW, &b.logV)) return QMC_ERR_UNSUPPORTED;
  b.logM = b.logW + b.logV;

  PassArgs c = base;
  c.LP = p.L1; c.nst = p.rad1.n; c.rbits = p.rad1.packed(); c.point_stride = p.L2; c.line_stride = 1; c.n_linegroups = p.L2;
  c.fwd = 0; c.inv = 1; c.mul = 0; c.twiddle = 0;
  if (choose_tile(c.LP, T, 8, c.n_linegroups, &c.logW, &c.logV)) return QMC_ERR_UNSUPPORTED;
  c.logM = c.logW + c.logV;
  specs[0] = PassSpec{a, first_load, ST_SCRATCH, s0};
  specs[1] = PassSpec{b, LD_SCRATCH, ST_SCRATCH, s0 + 1};
  specs[2] = PassSpec{c, LD_SCRATCH, last_store, s0 + 2};
  *n = 3;
  return QMC_OK;
}

// The spectral pass's arguments with the packed rows of the sparse first
// pass (b->sp_*), when the product takes that path: a forward product with
// 8-column panels whose plan chooses it (sparse_first_pass).
bool qmc::sparse_spectral_args(const Plan& p, int dir, const PassSpec* specs, int n, PassArgs* b) {
  if (!(n == 3 && dir > 0 && specs[0].load == LD_GATHER_A && specs[1].a.logW == 3 &&
        sparse_first_pass(p, specs[1].a.T)))
    return false;
  *b = specs[1].a;
  b->sp_pos = p.d_sp_pos;
  b->sp_row = p.d_sp_row;
  b->sp_gptr = p.d_sp_gptr;
  b->sp_s = p.s;
  b->sp_ap = static_cast<unsigned char*>(p.d_scratch) + work_bytes(p, b->T);
  return true;
}

namespace {

// True when the first pass would gather many rows per line: no padded
// gather table (some line holds more than kGatherMax rows) and at least one
// row per four positions on average.
bool dense_positions(const Plan& p) { return p.L2 > 1 && p.gp_em == 0 && 4 * (int64_t)p.s >= p.L; }

// Runs the forward product (dir = +1) or the adjoint (dir = -1); with
// stage >= 0 every pass is profiled under that stage.
int run_product(Plan& p, int dir, PassArgs base, cudaStream_t st, int stage = -1) {
  PassSpec specs[3];
  int n = 0, rc;
  if ((rc = product_passes(p, dir, base, specs, &n))) return rc;
  PassArgs b;
  if (sparse_spectral_args(p, dir, specs, n, &b)) {
    // few rows of A per line: pack them by panel, then let the spectral
    // pass sum each of its lines from them (no first pass, nothing of the
    // work array read)
    if ((rc = timed(p, stage >= 0 ? stage : QMC_STAGE_SPARSE_PACK, st, [&] { return launch_sparse_pack(b, st); })))
      return rc;
    rc = timed(p, stage >= 0 ? stage : QMC_STAGE_FWD_SPARSE, st, [&] { return launch_pipe_sparse(b, st); });
    if (rc == QMC_OK) {
      const PassSpec& sp = specs[2];
      return timed(p, stage >= 0 ? stage : sp.stage, st, [&] { return pass(p, sp.a, sp.load, sp.store, st); });
    }
    if (rc != QMC_ERR_UNSUPPORTED) return rc;
  }
  if (n == 3 && specs[0].load == LD_GATHER_A && dense_positions(p)) {
    // densely hit positions: stream P·A into the work array first, then the
    // first pass transforms it like any other
    if ((rc = timed(p, stage >= 0 ? stage : QMC_STAGE_DENSE_SCATTER, st,
                    [&] { return launch_dense_scatter(specs[0].a, st); })))
      return rc;
    specs[0].load = LD_SCRATCH;
  }
  for (int i = 0; i < n; ++i) {
    const PassSpec& sp = specs[i];
    if ((rc = timed(p, stage >= 0 ? stage : sp.stage, st, [&] { return pass(p, sp.a, sp.load, sp.store, st); })))
      return rc;
  }
  return QMC_OK;
}

}  // namespace

// Korobov p-set product (Section 2.2): the L blocks Y'_b = Z·P_b share Z,
// so they run as one product whose (L·t) real right-hand sides are the t
// columns of A under the L selectors; block b's output rows start at
// ps_blk[b]·L.
int pset_matmul(Plan& p, const void* A, int64_t lda, int t, int a_dtype, float* out, int64_t ldo,
                float* row_mean, double* exp_sum, const float* col_off, int out_exp, cudaStream_t st) {
  if (row_mean || exp_sum) return QMC_ERR_UNSUPPORTED;
  const int64_t tt = p.L * (int64_t)t;  // combined real columns
  if (tt > (int64_t)1 << 30) return QMC_ERR_SHAPE;
  int rc;
  if ((rc = ensure_stats(p, colstats_bytes(p.s, t)))) return rc;
  float *cscale = nullptr, *cinv = nullptr;
  if ((rc = timed(p, QMC_STAGE_ROW0, st, [&] {
         return launch_colstats(p.d_stats, A, lda, p.s, t, a_dtype == QMC_DTYPE_F64, 0, 1.f, 0.0, nullptr,
                                nullptr, nullptr, &cscale, &cinv, st, p.d_err);
       })))
    return rc;
  PassArgs base{};
  base.cscale = cscale;
  base.cinv = cinv;
  base.t = (int)tt;
  base.T = (int)((tt + 1) / 2);
  base.t_a = t;
  base.s_a = p.s;
  base.A = A; base.lda = lda; base.a_f64 = a_dtype == QMC_DTYPE_F64;
  base.out = out; base.ldo = ldo;
  base.ps_d = p.d_ps_d; base.ps_inv = p.d_ps_inv; base.ps_blk = p.d_ps_blk;
  base.inv_t = 1.0f;
  base.col_off = col_off; base.out_exp = out_exp;
  return run_product(p, +1, base, st);
}

// qmc_matmul and qmc_matmul_affine: B = Y·A with the optional epilogues
// (row mean, Σ exp, or the affine map col_off[k] + B then exp()).
int matmul_impl(void* plan, const void* A, int64_t lda, int32_t t, int32_t a_dtype, float* out, int64_t ldo,
                float* row_mean, double* exp_sum, const float* col_off, int out_exp, void* stream) {
  if (!plan || !A || !out) return QMC_ERR_INVALID;
  Plan& p = *static_cast<Plan*>(plan);
  if (t < 1 || lda < t || ldo < t) return QMC_ERR_SHAPE;
  if (a_dtype != QMC_DTYPE_F32 && a_dtype != QMC_DTYPE_F64) return QMC_ERR_INVALID;
  if (p.prec == QMC_PREC_FP32_SPLIT && a_dtype != QMC_DTYPE_F64) return QMC_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (p.pset) return pset_matmul(p, A, lda, t, a_dtype, out, ldo, row_mean, exp_sum, col_off, out_exp, st);
  if (row_mean && cudaMemsetAsync(row_mean, 0, sizeof(float) * p.out_rows, st) != cudaSuccess)
    return QMC_ERR_CUDA;
  if (exp_sum && cudaMemsetAsync(exp_sum, 0, sizeof(double), st) != cudaSuccess) return QMC_ERR_CUDA;
  int rc;
  if (p.L2 == 1 && !row_mean && p.prec == QMC_PREC_FP32 && p.pass_kernel == QMC_KERNEL_AUTO && t <= 16) {
    // small single-pass product: column statistics and the pass in one launch
    PassArgs base{};
    base.T = complex_columns(p, t);
    base.t = t;
    base.A = A; base.lda = lda; base.a_f64 = a_dtype == QMC_DTYPE_F64;
    base.a_vec2 = !base.a_f64 && (lda % 2 == 0) && aligned8(A);
    base.out = out; base.ldo = ldo; base.o_vec2 = (ldo % 2 == 0) && aligned8(out);
    base.inv_t = 1.0f / (float)t; base.exp_sum = exp_sum;
    base.col_off = col_off; base.out_exp = out_exp;
    PassSpec specs[3];
    int n = 0;
    if ((rc = product_passes(p, +1, base, specs, &n))) return rc;
    if (n == 1) {
      rc = timed(p, QMC_STAGE_FWD_FUSED, st, [&] { return launch_small_product(p, specs[0], st); });
      if (rc != QMC_ERR_UNSUPPORTED) return rc;
    }
  }
  if ((rc = ensure_stats(p, colstats_bytes(p.s, t)))) return rc;
  float *cscale = nullptr, *cinv = nullptr;
  if ((rc = timed(p, QMC_STAGE_ROW0, st, [&] {
         return launch_colstats(p.d_stats, A, lda, p.s, t, a_dtype == QMC_DTYPE_F64, 0, 1.f, p.phi0,
                                p.has_row0 ? out : nullptr, p.has_row0 ? row_mean : nullptr, exp_sum,
                                &cscale, &cinv, st, p.d_err);
       })))
    return rc;
  PassArgs base{};
  base.cscale = cscale;
  base.cinv = cinv;
  base.T = complex_columns(p, t);
  base.t = t;
  base.A = A; base.lda = lda; base.a_f64 = a_dtype == QMC_DTYPE_F64;
  base.split = p.prec == QMC_PREC_FP32_SPLIT;
  base.a_vec2 = !base.a_f64 && (lda % 2 == 0) && aligned8(A);
  base.out = out; base.ldo = ldo; base.o_vec2 = (ldo % 2 == 0) && aligned8(out);
  const bool fused_mean = row_mean && p.row_mean_mode == QMC_ROW_MEAN_FUSED;
  base.row_mean = fused_mean ? row_mean : nullptr;
  base.inv_t = 1.0f / (float)t; base.exp_sum = exp_sum;
  base.col_off = col_off; base.out_exp = out_exp;
  if ((rc = run_product(p, +1, base, st))) return rc;
  // row 0 came from the column statistics: apply the affine epilogue to it
  if (p.has_row0 && (col_off || out_exp) && (rc = launch_row0_affine(out, t, col_off, out_exp, st)))
    return rc;
  if (!row_mean || fused_mean) return QMC_OK;
  // Row mean by linearity: (1/t) Σ_k (Y A)_nk = (Y ā)_n with ā = A·1/t, one
  // more product of a single column (row 0 included through its column sum).
  if ((rc = timed(p, QMC_STAGE_ROW_MEAN, st, [&] {
         return launch_row_average(A, lda, p.s, t, a_dtype == QMC_DTYPE_F64, p.d_abar, st);
       })))
    return rc;
  float *cs1 = nullptr, *ci1 = nullptr;
  if ((rc = timed(p, QMC_STAGE_ROW_MEAN, st, [&] {
         return launch_colstats(p.d_stats, p.d_abar, 1, p.s, 1, a_dtype == QMC_DTYPE_F64, 0, 1.f, p.phi0,
                                p.has_row0 ? row_mean : nullptr, nullptr, nullptr, &cs1, &ci1, st, p.d_err);
       })))
    return rc;
  PassArgs one = base;
  one.cscale = cs1; one.cinv = ci1;
  one.T = 1; one.t = 1;
  one.A = p.d_abar; one.lda = 1; one.a_vec2 = 0;
  one.out = row_mean; one.ldo = 1; one.o_vec2 = 0;
  one.row_mean = nullptr; one.exp_sum = nullptr; one.inv_t = 1.f;
  one.col_off = nullptr; one.out_exp = 0;
  return run_product(p, +1, one, st, QMC_STAGE_ROW_MEAN);
}


extern "C" {

const char* qmc_status_string(int s) {
  switch (s) {
    case QMC_OK: return "ok";
    case QMC_ERR_INVALID: return "invalid argument";
    case QMC_ERR_NOT_PRIME: return "N is not prime (or not a power of two for F_2)";
    case QMC_ERR_NOT_PRIMITIVE: return "generator of the field is not primitive";
    case QMC_ERR_GENERATOR: return "invalid generating vector entry";
    case QMC_ERR_SHAPE: return "invalid matrix shape or leading dimension";
    case QMC_ERR_UNSUPPORTED: return "unsupported size (FFT length factorisation or range)";
    case QMC_ERR_ALLOC: return "device allocation failed";
    case QMC_ERR_CUDA: return "CUDA runtime error";
    case QMC_ERR_TIMEOUT: return "bounded device wait timed out";
    case QMC_ERR_DEVICE: return "error latched by a kernel";
    case QMC_ERR_SCRATCH: return "problem needs more scratch than the fixed no-alloc array holds";
    case QMC_ERR_NONFINITE: return "an input column held a NaN or an infinity";
    case QMC_ERR_BOUNDS: return "an index read from a plan table was out of range (QMC_CHECK_BOUNDS build)";
  }
  return "unknown status";
}

int qmc_version(void) { return 100; }

int64_t qmc_kernel_launches(void) { return (int64_t)qmc::launch_total(); }

int qmc_plan_set_option(void* plan, int32_t option, int64_t value) {
  if (!plan) return QMC_ERR_INVALID;
  Plan& p = *static_cast<Plan*>(plan);
  switch (option) {
    case QMC_OPT_PASS_KERNEL:
      if (value < QMC_KERNEL_AUTO || value > QMC_KERNEL_PIPELINED) return QMC_ERR_INVALID;
      p.pass_kernel = (int)value;
      return QMC_OK;
    case QMC_OPT_ROW_MEAN:
      if (value != QMC_ROW_MEAN_LINEAR && value != QMC_ROW_MEAN_FUSED) return QMC_ERR_INVALID;
      p.row_mean_mode = (int)value;
      return QMC_OK;
    case QMC_OPT_FIRST_PASS:
      if (value < QMC_FIRST_PASS_AUTO || value > QMC_FIRST_PASS_SPARSE) return QMC_ERR_INVALID;
      p.first_pass = (int)value;
      return QMC_OK;
    case QMC_OPT_FFT_SPLIT:
      return replan_split(p, value);
    default:
      return QMC_ERR_INVALID;
  }
}

int qmc_plan_set_profiling(void* plan, int32_t enable) {
  if (!plan) return QMC_ERR_INVALID;
  static_cast<Plan*>(plan)->profiling = enable ? 1 : 0;
  return QMC_OK;
}

int qmc_plan_read_profile(void* plan, double* ms, int32_t* launches) {
  if (!plan || !ms || !launches) return QMC_ERR_INVALID;
  Plan& p = *static_cast<Plan*>(plan);
  for (int i = 0; i < QMC_NUM_STAGES; ++i) { ms[i] = 0.0; launches[i] = 0; }
  int rc = QMC_OK;
  for (auto& m : p.marks) {
    float e = 0.f;
    if (cudaEventSynchronize(m.stop) != cudaSuccess || cudaEventElapsedTime(&e, m.start, m.stop) != cudaSuccess)
      rc = QMC_ERR_CUDA;
    if (m.stage >= 0 && m.stage < QMC_NUM_STAGES) { ms[m.stage] += e; launches[m.stage] += 1; }
    p.event_pool.push_back(m.start);
    p.event_pool.push_back(m.stop);
  }
  p.marks.clear();
  return rc;
}

int qmc_plan_create(void** out, const qmc_desc* d, void* stream) {
  if (!out) return QMC_ERR_INVALID;
  *out = nullptr;
  if (!d || d->s < 1 || (!d->gen_host && d->kind != QMC_KOROBOV_PSET)) return QMC_ERR_INVALID;
  if (d->map < 0 || d->map > QMC_MAP_TENT || d->row0 < 0 || d->row0 > QMC_ROW0_EXCLUDE ||
      d->order < 0 || d->order > QMC_ORDER_CIRCULANT || d->prec < 0 || d->prec > QMC_PREC_FP32_SPLIT)
    return QMC_ERR_INVALID;
  if (!(d->shift >= 0.0 && d->shift < 1.0)) return QMC_ERR_INVALID;  // also rejects NaN
  Plan* p = new (std::nothrow) Plan();
  if (!p) return QMC_ERR_ALLOC;
  p->kind = d->kind; p->N = d->N; p->s = d->s; p->map = d->map; p->row0 = d->row0;
  p->shift = d->shift;
  p->order = d->order; p->prec = d->prec; p->g = 0; p->P = 0; p->m = 0;
  if (d->kind == QMC_KOROBOV_PSET) {
    // The p-set's blocks are rank-1 lattices with prime K = N: the plan's
    // tables are those of the prime case, plus the per-block solvers.
    if (d->row0 == QMC_ROW0_INCLUDE || d->prec != QMC_PREC_FP32) { delete p; return QMC_ERR_INVALID; }
    p->pset = 1;
    p->kind = QMC_LATTICE_PRIME;
  }
  if (p->kind == QMC_LATTICE_PRIME) {
    if (d->N < 3 || d->N >= (int64_t(1) << 31) || !is_prime_u64(d->N)) { delete p; return QMC_ERR_NOT_PRIME; }
    p->L = d->N - 1;
    if (d->g == 0) {
      for (int64_t g = 2; g < d->N; ++g)
        if (is_primitive_root(g, d->N)) { p->g = g; break; }
    } else {
      if (!is_primitive_root(d->g, d->N)) { delete p; return QMC_ERR_NOT_PRIMITIVE; }
      p->g = d->g;
    }
  } else if (p->kind == QMC_LATTICE_F2) {
    int m = 0;
    while ((int64_t(1) << m) < d->N) ++m;
    if (d->N < 4 || (int64_t(1) << m) != d->N || m > 30) { delete p; return QMC_ERR_NOT_PRIME; }
    p->m = m;
    p->L = d->N - 1;
    if (d->modulus_P == 0) {
      for (uint64_t P = (uint64_t(1) << m) + 1; P < (uint64_t(1) << (m + 1)); P += 2)
        if (f2_is_primitive(P, m)) { p->P = P; break; }
    } else {
      if (!f2_is_primitive(d->modulus_P, m)) { delete p; return QMC_ERR_NOT_PRIMITIVE; }
      p->P = d->modulus_P;
    }
    if (!p->P) { delete p; return QMC_ERR_NOT_PRIMITIVE; }
    p->base = 2;
  } else if (p->kind == QMC_LATTICE_FB) {
    const int b = d->base;
    if (b < 2 || b >= 256 || !is_prime_u64(b)) { delete p; return QMC_ERR_NOT_PRIME; }
    int m = 0;
    int64_t bm = 1;
    while (bm < d->N && bm < (int64_t(1) << 31)) { bm *= b; ++m; }
    if (d->N < 4 || bm != d->N || d->N >= (int64_t(1) << 31)) { delete p; return QMC_ERR_NOT_PRIME; }
    p->m = m;
    p->base = b;
    p->L = d->N - 1;
    if (d->modulus_P == 0) {
      for (uint64_t P = (uint64_t)bm + 1; P < 2 * (uint64_t)bm; ++P)
        if (fb_is_primitive(P, b, m, p->L)) { p->P = P; break; }
    } else {
      if (!fb_is_primitive(d->modulus_P, b, m, p->L)) { delete p; return QMC_ERR_NOT_PRIMITIVE; }
      p->P = d->modulus_P;
    }
    if (!p->P) { delete p; return QMC_ERR_NOT_PRIMITIVE; }
  } else {
    delete p;
    return QMC_ERR_INVALID;
  }
  if (p->shift == 0.0) {
    p->phi0 = phi_at_zero(d->map);
  } else {
    // the row-0 point is {0 + Δ} = Δ; φ(Δ) from the device routine that
    // evaluates the generator sequence
    const int mrc = map_value(d->map, p->shift, &p->phi0, (cudaStream_t)stream);
    if (mrc != QMC_OK) { delete p; return mrc; }
  }
  if (d->row0 == QMC_ROW0_AUTO) p->has_row0 = isfinite(p->phi0) ? 1 : 0;
  else if (d->row0 == QMC_ROW0_INCLUDE) {
    if (!isfinite(p->phi0)) { delete p; return QMC_ERR_INVALID; }
    p->has_row0 = 1;
  } else p->has_row0 = 0;
  if (p->pset) p->has_row0 = 0;  // n, γ >= 1: no zero point
  p->out_rows = p->has_row0 ? p->N : p->N - 1;
  if (p->pset) p->out_rows = p->L * p->L;
  if (!choose_factorisation(p->L, *p)) { delete p; return QMC_ERR_UNSUPPORTED; }
  int rc;
  if (p->pset) {
    // tables for the block b = 1 exponents e_j = j mod L (plain lattice
    // tables; the p-set product itself uses the per-block solvers)
    std::vector<int64_t> e1((size_t)p->s);
    for (int j = 0; j < p->s; ++j) e1[(size_t)j] = j % p->L;
    rc = build_tables(*p, e1.data(), 1, (cudaStream_t)stream);
    if (rc == QMC_OK) rc = build_pset_tables(*p, (cudaStream_t)stream);
  } else {
    rc = build_tables(*p, d->gen_host, d->gen_is_exponent, (cudaStream_t)stream);
  }
  if (rc != QMC_OK) { free_plan(p); return rc; }
  *out = p;
  return QMC_OK;
}

int qmc_plan_destroy(void* plan) {
  if (!plan) return QMC_ERR_INVALID;
  cudaDeviceSynchronize();
  free_plan(static_cast<Plan*>(plan));
  return QMC_OK;
}

int qmc_plan_info(void* plan, qmc_info* info) {
  if (!plan || !info) return QMC_ERR_INVALID;
  const Plan& p = *static_cast<Plan*>(plan);
  memset(info, 0, sizeof(*info));
  info->N = p.N; info->L = p.L; info->g = p.g; info->modulus_P = p.P; info->s = p.s;
  info->n_distinct = p.n_distinct;
  info->collision_adds = p.s - p.n_distinct;
  info->row0_adds = (p.has_row0 && p.phi0 != 0.0) ? p.s - 1 : 0;
  info->out_rows = p.out_rows; info->phi0 = p.phi0;
  info->base = p.base;
  info->L1 = p.L1; info->L2 = p.L2; info->has_row0 = p.has_row0;
  return QMC_OK;
}

int qmc_plan_exponents(void* plan, int32_t* e_host) {
  if (!plan || !e_host) return QMC_ERR_INVALID;
  const Plan& p = *static_cast<Plan*>(plan);
  memcpy(e_host, p.e_host.data(), sizeof(int32_t) * p.s);
  return QMC_OK;
}

int qmc_plan_copy_table(void* plan, int32_t which, void* dst, int64_t bytes) {
  if (!plan || !dst) return QMC_ERR_INVALID;
  const Plan& p = *static_cast<Plan*>(plan);
  const void* src = nullptr;
  int64_t need = 0;
  switch (which) {
    case QMC_TABLE_POW: src = p.d_pow; need = 4 * p.L; break;
    case QMC_TABLE_LOG: src = p.d_log; need = 4 * p.log_size; break;
    case QMC_TABLE_EXPONENTS: src = p.d_e; need = 4 * (int64_t)p.s; break;
    case QMC_TABLE_OUT_ROW: src = p.d_orow; need = 4 * p.L; break;
    case QMC_TABLE_ZETA: src = p.d_zeta; need = 8 * p.L; break;
    case QMC_TABLE_SPECTRUM64: src = p.d_H64; need = 16 * p.L; break;
    case QMC_TABLE_ROW_PTR: src = p.d_row_ptr; need = 4 * (p.L + 1); break;
    case QMC_TABLE_JLIST: src = p.d_jlist; need = 4 * (int64_t)p.s; break;
    default: return QMC_ERR_INVALID;
  }
  if (bytes != need) return QMC_ERR_SHAPE;
  return cudaMemcpy(dst, src, (size_t)bytes, cudaMemcpyDeviceToHost) == cudaSuccess ? QMC_OK
                                                                                   : QMC_ERR_CUDA;
}

#ifdef QMC_CHECK_BOUNDS
int qmc_debug_poke_table(void* plan, int32_t which, int64_t index, int32_t value, int32_t* old) {
  if (!plan || !old) return QMC_ERR_INVALID;
  Plan& p = *static_cast<Plan*>(plan);
  int* t = nullptr;
  int64_t n = 0;
  switch (which) {
    case QMC_TABLE_OUT_ROW: t = p.d_orow; n = p.L; break;
    case QMC_TABLE_JLIST: t = p.d_jlist; n = p.s; break;
    default: return QMC_ERR_INVALID;
  }
  if (!t || index < 0 || index >= n) return QMC_ERR_SHAPE;
  if (cudaMemcpy(old, t + index, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(t + index, &value, sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return QMC_ERR_CUDA;
  return QMC_OK;
}
#endif

int qmc_plan_reserve(void* plan, int32_t t_max) {
  if (!plan || t_max < 1) return QMC_ERR_INVALID;
  Plan& p = *static_cast<Plan*>(plan);
  const int rc = ensure_stats(p, colstats_bytes((int)std::max<int64_t>(p.s, p.out_rows), t_max));
  if (rc) return rc;
  return ensure_scratch(p, scratch_need(p, t_max));
}

int qmc_plan_sync_status(void* plan, void* stream) {
  if (!plan) return QMC_ERR_INVALID;
  Plan& p = *static_cast<Plan*>(plan);
  int h = 0;
  if (cudaMemcpyAsync(&h, p.d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return QMC_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return QMC_ERR_CUDA;
  if (h) {
    cudaMemsetAsync(p.d_err, 0, sizeof(int), (cudaStream_t)stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    if (h & kErrBounds) return QMC_ERR_BOUNDS;
    if (h & kErrTimeout) return QMC_ERR_TIMEOUT;
    if (h & kErrGenerator) return QMC_ERR_GENERATOR;
    if (h & kErrNonFinite) return QMC_ERR_NONFINITE;
    return QMC_ERR_DEVICE;
  }
  return QMC_OK;
}

int qmc_matmul(void* plan, const void* A, int64_t lda, int32_t t, int32_t a_dtype, float* out,
               int64_t ldo, float* row_mean, double* exp_sum, void* stream) {
  return matmul_impl(plan, A, lda, t, a_dtype, out, ldo, row_mean, exp_sum, nullptr, 0, stream);
}

int qmc_matmul_affine(void* plan, const void* A, int64_t lda, int32_t t, int32_t a_dtype,
                      const float* col_offset, int32_t apply_exp, float* out, int64_t ldo, void* stream) {
  if (apply_exp != 0 && apply_exp != 1) return QMC_ERR_INVALID;
  return matmul_impl(plan, A, lda, t, a_dtype, out, ldo, nullptr, nullptr, col_offset, apply_exp, stream);
}

int qmc_matmul_backward(void* plan, const float* G, int64_t ldg, int32_t t, int32_t g_mode,
                        float* dA, int64_t ldda, void* stream) {
  if (!plan || !G || !dA) return QMC_ERR_INVALID;
  Plan& p = *static_cast<Plan*>(plan);
  if (p.pset) return QMC_ERR_UNSUPPORTED;
  if (t < 1 || ldg < t || ldda < t) return QMC_ERR_SHAPE;
  if (g_mode != 0 && g_mode != 1) return QMC_ERR_INVALID;
  PassArgs base{};
  base.T = (t + 1) / 2;   // the adjoint always pairs FP32 columns
  base.t = t;
  base.G = G; base.ldg = ldg; base.g_vec2 = (ldg % 2 == 0) && aligned8(G);
  base.g_exp = g_mode; base.g_scale = (float)(1.0 / ((double)p.out_rows * (double)t));
  base.dA = dA; base.ldda = ldda; base.d_vec2 = (ldda % 2 == 0) && aligned8(dA);
  base.has_row0 = p.has_row0; base.phi0 = (float)p.phi0; base.row0_out = 0;
  int rc0;
  if ((rc0 = ensure_stats(p, colstats_bytes((int)p.out_rows, t)))) return rc0;
  float *cscale = nullptr, *cinv = nullptr;
  if ((rc0 = timed(p, QMC_STAGE_ROW0, (cudaStream_t)stream, [&] {
         return launch_colstats(p.d_stats, G, ldg, (int)p.out_rows, t, 0, g_mode, base.g_scale, 0.0,
                                nullptr, nullptr, nullptr, &cscale, &cinv, (cudaStream_t)stream, p.d_err);
       })))
    return rc0;
  base.cscale = cscale;
  base.cinv = cinv;
  const int saved = p.prec;
  p.prec = QMC_PREC_FP32;  // scratch sizing for paired columns
  const int rc = run_product(p, -1, base, (cudaStream_t)stream);
  p.prec = saved;
  return rc;
}

int qmc_generate_points(void* plan, float* Y, int64_t ldy, void* stream) {
  if (!plan || !Y) return QMC_ERR_INVALID;
  const Plan& p = *static_cast<Plan*>(plan);
  if (ldy < p.s) return QMC_ERR_SHAPE;
  return launch_generate_points(p, Y, ldy, (cudaStream_t)stream);
}

}  // extern "C"

// Forward-product prologue shared with the batch: column statistics (and
// row 0) on `st`, and the input/output fields of the pass arguments.
int qmc::forward_prologue(Plan& p, const void* A, int64_t lda, int t, int a_dtype, float* out,
                          int64_t ldo, cudaStream_t st, PassArgs* base, ColstatsJob* defer) {
  int rc;
  if ((rc = ensure_stats(p, colstats_bytes(p.s, t)))) return rc;
  float *cscale = nullptr, *cinv = nullptr;
  if (defer) {
    if (a_dtype != QMC_DTYPE_F32) return QMC_ERR_UNSUPPORTED;
    colstats_job(p.d_stats, static_cast<const float*>(A), lda, p.s, t, p.phi0, p.has_row0 ? out : nullptr, p.d_err,
                 defer, &cscale, &cinv);
  } else if ((rc = launch_colstats(p.d_stats, A, lda, p.s, t, a_dtype == QMC_DTYPE_F64, 0, 1.f, p.phi0,
                                   p.has_row0 ? out : nullptr, nullptr, nullptr, &cscale, &cinv, st, p.d_err))) {
    return rc;
  }
  *base = PassArgs{};
  base->cscale = cscale;
  base->cinv = cinv;
  base->T = complex_columns(p, t);
  base->t = t;
  base->A = A; base->lda = lda; base->a_f64 = a_dtype == QMC_DTYPE_F64;
  base->split = p.prec == QMC_PREC_FP32_SPLIT;
  base->a_vec2 = !base->a_f64 && (lda % 2 == 0) && aligned8(A);
  base->out = out; base->ldo = ldo; base->o_vec2 = (ldo % 2 == 0) && aligned8(out);
  base->inv_t = 1.0f / (float)t;
  return QMC_OK;
}

// One FP32 pass with the plan's kernel choice (used by the batch graph).
int qmc::launch_plan_pass(const Plan& p, const PassSpec& sp, cudaStream_t st) {
  return pass(p, sp.a, sp.load, sp.store, st);
}
