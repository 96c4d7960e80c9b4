// qmc_internal.h — plan object and pass descriptors shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/qmc.h"
#include "fft_engine.cuh"

namespace qmc {

// Largest per-line entry count of the padded first-pass gather table.
constexpr int kGatherMax = 32;
// First-pass lines with at most this many entries take their DFT term by
// term instead of the transform.
constexpr int kDirectEntries = 4;

// Error bits latched in the plan's device error word.
enum : int {
  kErrGenerator = 1,    // z_j ≡ 0, q_j out of range, e_j out of [0, L)
  kErrNotPrimitive = 2, // power table is not a bijection
  kErrBounds = 4,       // an index check failed inside a kernel
  kErrTimeout = 8,      // a bounded wait gave up
  kErrNonFinite = 16    // a column of the input holds a NaN or an infinity
};

// Index check of the QMC_CHECK_BOUNDS build: an index read from a plan
// table (a row of A, of B or of G, a point of a line) outside [0, n)
// latches kErrBounds in the error word and is replaced by 0, so that the
// access stays inside its buffer (no trap); the call's status then reports
// QMC_ERR_BOUNDS and its output is not valid.  Without the flag the check
// compiles to nothing.
template <typename I>
__device__ __forceinline__ I chk(I i, int64_t n, int* err) {
#ifdef QMC_CHECK_BOUNDS
  if ((uint64_t)(int64_t)i >= (uint64_t)n) {
    if (err) atomicOr(err, kErrBounds);
    return I(0);
  }
#else
  (void)n;
  (void)err;
#endif
  return i;
}

enum LoadMode : int {
  LD_SCRATCH = 0,   // previous pass's output
  LD_GATHER_A = 1,  // scatter-add a'_u = sum_{e_j = u} A_j (forward first pass)
  LD_PERM_G = 2,    // g'_r = G[out_row(r)] (adjoint first pass)
  LD_DENSE64 = 3,   // a real FP64 vector (plan-time spectrum)
  LD_PSET = 4       // p-set: a'_{b,u} = Σ_{j b = u mod L} A_j for right-hand side block b
};

enum StoreMode : int {
  ST_SCRATCH = 0,   // next pass's input
  ST_OUT = 1,       // out[out_row(r)] with epilogues (forward last pass)
  ST_DA = 2,        // dA[j] for every j with e_j = r (adjoint last pass)
  ST_PSET = 3       // p-set: out[rowblock(b) + out_row(r)] for right-hand side block b
};

// Geometry and operands of one pass over the L x T (complex) work array.
// Work array layout ("panels"): panel p holds complex columns
// [p*W, p*W + W); element (row r, column p*W + w) is at
// scratch[(p*L + r)*W + w].  A pass transforms LP points of each line;
// point i of line group a is row r = a*line_stride + i*point_stride.
struct PassArgs {
  int L;
  int LP;
  int nst;                // number of radix stages of the LP-point FFT
  uint64_t rbits;         // their radices, 5 bits each (Radices::packed)
  int logW, logV, logM;   // W columns x V line groups = M lines per tile
  int point_stride;
  int line_stride;
  int n_linegroups;
  int T;                  // complex columns
  int fwd, inv;           // apply forward / inverse transform
  int twiddle;            // 0, -1 (forward sign) or +1: multiply by w_L^{+-a*i}
  int mul;                // 0 none, 1 spectrum H, 2 conj(H)
  void* scratch;
  const void* H;          // cx<R>[L], in the order the inner pass consumes
  const void* twL;        // cx<R>[L]: exp(+2 pi i k / L)
  // inputs
  const void* A; int64_t lda; int t; int a_f64; int split; int a_vec2;
  const int* row_ptr; const int* jlist; const int* orow;
  const int* bucket_ptr; const int* blist;   // non-empty points per first-pass line
  const int* gp_i; const int* gp_j; int gp_em;  // padded gather table (gp_em = 0: none)
  // first-pass lines split by entry count (P x Q first pass): n_pair line
  // pairs (2λ, 2λ+1, by their first line) and n_direct single lines with at
  // most kDirectEntries entries each, then n_fft lines with more
  const int* lines; int n_pair, n_direct, n_fft;
  const float* G; int64_t ldg; int g_exp; float g_scale; int g_vec2;
  const double* zeta;
  // outputs
  float* out; int64_t ldo; int o_vec2;
  float* row_mean; float inv_t;
  double* exp_sum;
  // affine output epilogue (qmc_matmul_affine): out = col_off[k] + value,
  // then exp() when out_exp (Sections 3.2 and 3.3)
  const float* col_off; int out_exp;
  float* dA; int64_t ldda; int d_vec2;
  int has_row0; float phi0; int row0_out;  // adjoint: + phi0 * G[row0_out]
  const void* rader;      // cx<R>[768]: tw256, what_fwd, what_inv (Rader-257 passes)
  const int16_t* rader_perm;  // [512]: pin, pout
  // per real column: power-of-two scale applied on load and its inverse
  // applied on store (0 for a zero column); global memory, or shared memory
  // in the single-launch small product, so read them with generic loads in
  // code that kernel shares (pass_tile and qmc_io.cuh)
  const float* cscale;
  const float* cinv;
  int* err;
  int64_t n_out;          // rows of B (and of G): bound of the out-row table
  // Korobov p-set (LD_PSET / ST_PSET): real column q of the combined
  // problem is column q % t_a of right-hand side block b = q / t_a
  int t_a;                // columns of A
  int s_a;                // rows of A
  const int* ps_d;        // [L] gcd(b, L) (L for b = 0)
  const int* ps_inv;      // [L] (b / d)^{-1} mod (L / d)
  const int* ps_blk;      // [L] first output row of block b, divided by L
  // sparse first pass (QMC_FIRST_PASS_SPARSE): the rows of A as entries
  // q = 0..s-1 grouped by n2 mod P (group g at [sp_gptr[g], sp_gptr[g+1]))
  const int* sp_pos;      // [s] (n1 << 16) | n2 of the entry's position e = n1·L2 + n2
  const int* sp_row;      // [s] row j of A
  const int* sp_gptr;     // [P + 1]
  void* sp_ap;            // cx<float>[npan][s][8]: scaled column pairs of row sp_row[q]
  int sp_s;               // entries (= s)
};

struct Plan {
  // descriptor
  int kind;
  int64_t N;
  int64_t L;
  int64_t g;
  uint64_t P;     // F_2: bit i = coefficient of x^i; F_b: Σ p_i b^i
  int m;
  int base = 0;   // b of a polynomial lattice over F_b (2 for F_2), 0 for prime N
  int s;
  int map;
  int row0;
  int order;
  int prec;
  int has_row0;
  double shift;   // diagonal shift Δ (Remark 2)
  double phi0;    // φ at the row-0 point {0 + Δ} = Δ
  int64_t out_rows;
  int n_distinct;
  int L1, L2;
  Radices rad1, rad2;
  // device tables
  int* d_pow = nullptr;      // [L]
  int* d_log = nullptr;      // [log_size]
  int64_t log_size = 0;
  int* d_e = nullptr;        // [s]
  int* d_row_ptr = nullptr;  // [L+1]
  int* d_jlist = nullptr;    // [s]
  // distinct positions u grouped by first-pass line (u mod L2; one group
  // when L2 = 1), each group sorted by u: group b is
  // blist[bucket_ptr[b] .. bucket_ptr[b+1])
  int* d_bucket_ptr = nullptr;  // [L2 + 1]
  int* d_blist = nullptr;       // [s]
  // padded gather table of the first pass (multi-pass plans whose lines
  // hold at most kGatherMax j's): line b's entries at [b*gp_em, b*gp_em +
  // count), sorted by point index; point -1 marks padding
  int gp_em = 0;
  int* d_gp_i = nullptr;        // [L2 * gp_em] point index within the line
  int* d_gp_j = nullptr;        // [L2 * gp_em] row j of A
  // the first-pass lines ordered as [first lines of neighbouring pairs
  // with at most kDirectEntries entries each | other lines with at most
  // kDirectEntries entries | the others] (plans with a gather table)
  int* d_lines = nullptr;       // [L2]
  int n_pair = 0, n_direct = 0, n_fft = 0;
  int* d_orow = nullptr;     // [L]
  double* d_zeta = nullptr;  // [L]
  cx<float>* d_H = nullptr;  // [L]
  cx<double>* d_H64 = nullptr;  // [L]
  cx<float>* d_tw = nullptr;    // [L]
  // Rader-257 tables (only when a factor of L is 257): FP32 and FP64
  // copies of [tw256 | what_fwd | what_inv] and the int16 permutations.
  cx<float>* d_rader32 = nullptr;
  cx<double>* d_rader64 = nullptr;
  int16_t* d_rader_perm = nullptr;
  int* d_err = nullptr;
  // scratch
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  void* d_stats = nullptr;     // column statistics work area
  size_t stats_bytes = 0;
  std::vector<int32_t> e_host;
  int pass_kernel = QMC_KERNEL_AUTO;   // qmc_plan_set_option(QMC_OPT_PASS_KERNEL)
  int row_mean_mode = QMC_ROW_MEAN_LINEAR;
  // Korobov p-set plans: per right-hand side block b = 0..L-1
  int pset = 0;
  int* d_ps_d = nullptr;
  int* d_ps_inv = nullptr;
  int* d_ps_blk = nullptr;
  void* d_abar = nullptr;              // [s] doubles: A·1/t for the linear row mean
  // sparse first pass tables (plans whose second pass has length 256 or
  // 1024; sp_P = sqrt(L2), 0 = none)
  int sp_P = 0;
  int* d_sp_pos = nullptr;
  int* d_sp_row = nullptr;
  int* d_sp_gptr = nullptr;
  int first_pass = QMC_FIRST_PASS_AUTO;   // qmc_plan_set_option(QMC_OPT_FIRST_PASS)
  // optional per-stage event timing (qmc_plan_set_profiling)
  int profiling = 0;
  struct Mark { int stage; cudaEvent_t start, stop; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;   // events reused by later profiled launches
};

// Devices the per-device caches below (and the no-allocation scratch
// address) cover; a call on a device with a higher ordinal gets QMC_ERR_CUDA.
constexpr int kMaxDevices = 64;

// Launch set-up of one kernel instantiation, kept per device: the dynamic
// shared memory it has been opted in to and its occupancy.
struct KernelSetup {
  std::mutex mu;
  size_t smem_ok[kMaxDevices] = {};    // opted-in dynamic shared memory (0: the 48 KB default)
  size_t occ_smem[kMaxDevices] = {};   // shared memory the occupancy was computed for
  int occ_threads[kMaxDevices] = {};
  int blocks_per_sm[kMaxDevices] = {};
  int sms[kMaxDevices] = {};
};

// Opts `kernel` in to `smem` bytes of dynamic shared memory on the current
// device (needed above 48 KB) and, when grid_cap is not null, sets
// *grid_cap = SMs × resident blocks of `threads` threads at that size (the
// grid of a persistent launch).  The set-up is kept per device and updated
// under a lock, so host threads that launch on different devices each
// configure their own.  A refusal leaves no pending CUDA error behind and
// returns QMC_ERR_UNSUPPORTED; a device ordinal of kMaxDevices or more
// returns QMC_ERR_CUDA.
template <typename K>
int setup_kernel(K kernel, KernelSetup& ks, size_t smem, int threads, int* grid_cap) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return QMC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(ks.mu);
  if (smem > 48 * 1024 && smem > ks.smem_ok[dev]) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return QMC_ERR_UNSUPPORTED;
    }
    ks.smem_ok[dev] = smem;
  }
  if (grid_cap) {
    if (!ks.blocks_per_sm[dev] || ks.occ_smem[dev] != smem || ks.occ_threads[dev] != threads) {
      int sms = 0, per_sm = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        return QMC_ERR_UNSUPPORTED;
      }
      ks.sms[dev] = sms;
      ks.blocks_per_sm[dev] = per_sm;
      ks.occ_smem[dev] = smem;
      ks.occ_threads[dev] = threads;
    }
    *grid_cap = ks.sms[dev] * ks.blocks_per_sm[dev];
  }
  return QMC_OK;
}

// Kernel launches on the product paths since load (qmc_kernel_launches).
void count_launch();
unsigned long long launch_total();
void add_launches(long long delta);  // graph capture/replay bookkeeping

// Host helpers implemented in qmc_passes.cu
int launch_pass(const PassArgs& a, int R_is_double, int load, int store, cudaStream_t st);
int choose_tile(int LP, int T, int elem_bytes, int n_linegroups, int* logW, int* logV);
bool factor_radices(int LP, Radices* out);
// Column sums / l1 norms -> power-of-two column scales (and row 0 of the
// forward product when out_row0 is given); qmc_colstats.cu.
size_t colstats_bytes(int rows, int t);
// abar = A·1/t (row averages of A), in A's element type
int launch_row_average(const void* A, int64_t lda, int s, int t, int a_f64, void* abar, cudaStream_t st);
int launch_colstats(void* work, const void* X, int64_t ldx, int rows, int t, int x_f64, int x_exp,
                    float x_scale, double phi0, float* out_row0, float* row_mean0, double* exp_sum,
                    float** scale_out, float** inv_out, cudaStream_t st, int* err = nullptr);
// One problem of a column-statistics launch over many problems (FP32
// input, row 0 kept when out_row0 is given, no epilogue terms): the layout
// launch_colstats uses in its work buffer, and each stage's first block.
struct ColstatsJob {
  const float* X;
  int64_t ldx;
  int rows, t, chunk_rows, chunks;
  double* part_sum;
  double* part_l1;
  float* scale;
  float* inv;
  double phi0;
  float* out_row0;
  int* err;
  int blocks_partial, blocks_final;  // blocks of the job in each stage
  int blk_partial, blk_final;        // its first block in each launch (set by the caller)
};
void colstats_job(void* work, const float* X, int64_t ldx, int rows, int t, double phi0, float* out_row0,
                  int* err, ColstatsJob* job, float** scale_out, float** inv_out);
// Both stages of `njobs` jobs (device memory) in two launches.
int launch_colstats_multi(const ColstatsJob* jobs, int njobs, int partial_blocks, int final_blocks,
                          cudaStream_t st);
int launch_generate_points(const Plan& p, float* Y, int64_t ldy, cudaStream_t st);
// a' = P·A streamed into the work array (densely hit positions; qmc_colstats.cu)
int launch_dense_scatter(const PassArgs& a, cudaStream_t st);
// out[k] = col_off[k] + out[k], then exp() (row 0 of qmc_matmul_affine)
int launch_row0_affine(float* out_row0, int t, const float* col_off, int out_exp, cudaStream_t st);

// Register-resident kernels for LP = 256, 1024 (qmc_fastpass.cu)
bool fast_pass_supported(int LP);
int launch_fast_pass(PassArgs a, int load, int store, cudaStream_t st);
// Register kernels for single-transform passes of length P·Q (qmc_pqpass.cu)
bool pq_pass_supported(int LP);
int launch_pq_pass(const PassArgs& a, int load, int store, cudaStream_t st);
// Register spectral pass of length 257 by Rader's algorithm (qmc_rader.cu)
int launch_rader_spectral(const PassArgs& a, int load, int store, cudaStream_t st);
// Persistent double-buffered variant for work-array passes (qmc_pipepass.cu)
int launch_pipe_pass(const PassArgs& a, int load, int store, cudaStream_t st);
int launch_pipe_gather(const PassArgs& a, cudaStream_t st);
// Sparse first pass folded into the spectral pass (qmc_pipepass.cu): the
// scaled column pairs of A's rows in entry order, then the spectral pass
// that sums each line from them
int launch_sparse_pack(const PassArgs& b, cudaStream_t st);
int launch_pipe_sparse(const PassArgs& b, cudaStream_t st);
// Persistent double-buffered P x Q passes, LP = 768 or 255 (qmc_pqpipe.cu)
int launch_pqpipe_pass(const PassArgs& a, int load, int store, cudaStream_t st);
int launch_pqpipe_spectral(const PassArgs& a, int load, int store, cudaStream_t st);

// One pass of a product: its arguments, load/store modes and profiling stage.
struct PassSpec {
  PassArgs a;
  int load, store, stage;
};
// Fills the FFT passes of a forward product (dir = +1) or adjoint (dir = -1)
// of `p` on input described by `base` (qmc_api.cu); allocates plan scratch.
int product_passes(Plan& p, int dir, PassArgs base, PassSpec* specs, int* n);
// The spectral pass's arguments for the sparse first pass when a forward
// product (dir = +1) with these passes takes it; false otherwise.
bool sparse_spectral_args(const Plan& p, int dir, const PassSpec* specs, int n, PassArgs* b);
// Column statistics of A on `st` and the I/O fields of the pass arguments.
// With `defer` (FP32 A only) the statistics are described there for a
// launch over many problems instead of launched.
int forward_prologue(Plan& p, const void* A, int64_t lda, int t, int a_dtype, float* out,
                     int64_t ldo, cudaStream_t st, PassArgs* base, ColstatsJob* defer = nullptr);
// Whole forward product of a small single-pass plan in one launch
// (qmc_small.cu); QMC_ERR_UNSUPPORTED sends the caller to the general path.
int launch_small_product(const Plan& p, const PassSpec& sp, cudaStream_t st);
// One pass launched with the plan's kernel choice.
int launch_plan_pass(const Plan& p, const PassSpec& sp, cudaStream_t st);

// Plan-table kernels (qmc_tables.cu)
int build_tables(Plan& p, const int64_t* gen_host, int gen_is_exponent, cudaStream_t st);
// φ(x) evaluated on the device by the same routine as the generator
// sequence (synchronous on st).
int map_value(int map, double x, double* out, cudaStream_t st);

}  // namespace qmc
