/*
 * qmc.h — C ABI of libqmcfft, the GB300 (sm_103a) fast QMC matrix product.
 *
 * The library computes B = Y·A where the rows of Y are the N points of a
 * rank-1 lattice rule (prime N) or of a polynomial lattice rule over F_2
 * (N = 2^m), each coordinate mapped by one univariate map φ, and A is any
 * s x t real matrix (Dick, Kuo, Le Gia, Schwab, "Fast QMC matrix-vector
 * multiplication", Section 1 and Section 2.1).
 *
 * Method (Section 2.1, Eq. (3)): with beta = g a primitive root of Z_N^*
 * and z_j = g^{e_j} mod N, the rows y_1..y_{N-1}, reordered by powers of
 * g^{-1}, factor as Y' = Z·P with Z the (N-1)-circulant of the generator
 * sequence z_k = φ({g^k/N}) and P the 0/1 selector with p_{e_j, j} = 1.
 * Y'·A is then a scatter-add of A's rows (P·A), a batched FFT of length
 * L = N-1 down the columns, a pointwise product with the once-computed
 * spectrum of z_k, an inverse FFT and an un-permute back to the
 * conventional row order; row 0 is y_0·a = φ(0)·Σ_j a_j.  Remark 1 extends
 * this to polynomial lattice rules (here over F_2 with a primitive modulus
 * P(x) and q_j = x^{e_j} mod P, L = 2^m - 1).
 *
 * Conventions for every entry point
 *   - Matrices are row-major with an explicit leading dimension (elements).
 *   - Pointers named A, out, G, dA, Y, row_mean, exp_sum are DEVICE
 *     pointers owned by the caller.  Pointers named *_host are host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).
 *     Calls are asynchronous on that stream unless stated otherwise.
 *   - Every call returns a qmc_status (0 = QMC_OK).  Nothing aborts.
 *     Errors detected inside kernels (invalid generator, a non-finite input
 *     column) are latched in the plan's device error word and returned by
 *     the next qmc_plan_sync_status().
 *   - A plan may be used by one stream at a time.  Plan-internal tables
 *     and scratch are owned by the plan and freed by qmc_plan_destroy().
 */
#ifndef QMC_H_
#define QMC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QMC_OK = 0,
  QMC_ERR_INVALID = 1,        /* null pointer, bad enum, bad size */
  QMC_ERR_NOT_PRIME = 2,      /* N is not prime (prime kind), not 2^m (F_2 kind), or b not prime / N not b^m (F_b kind) */
  QMC_ERR_NOT_PRIMITIVE = 3,  /* g is not a primitive root / P is not primitive */
  QMC_ERR_GENERATOR = 4,      /* z_j ≡ 0 mod N, q_j = 0, or e_j out of [0, L-1] */
  QMC_ERR_SHAPE = 5,          /* t < 1, ld too small */
  QMC_ERR_UNSUPPORTED = 6,    /* L has a prime factor outside {2,3,5,7,11,13,17,257}, N >= 2^31,
                                 or a call that a Korobov p-set plan does not offer */
  QMC_ERR_ALLOC = 7,          /* device allocation failed */
  QMC_ERR_CUDA = 8,           /* a CUDA runtime call failed */
  QMC_ERR_TIMEOUT = 9,        /* a bounded device wait gave up (batched launch) */
  QMC_ERR_DEVICE = 10,        /* an error latched by a kernel (see qmc_plan_sync_status) */
  QMC_ERR_SCRATCH = 11,       /* qmc_matmul_noalloc: the problem needs more scratch than
                                 the library's fixed array holds */
  QMC_ERR_NONFINITE = 12,     /* latched: a column of A (or of G, or exp(B) in the exp-loss
                                 adjoint) held a NaN or an infinity; the outputs of that
                                 column, and of the column it is paired with in one complex
                                 FFT column, are not finite */
  QMC_ERR_BOUNDS = 13         /* latched, QMC_CHECK_BOUNDS builds only: an index read from a
                                 plan table (a row of A, B or G, a point of a line) was out of
                                 range; the access went to index 0 instead and the outputs
                                 of the call are not valid */
} qmc_status;

/* QMC_KOROBOV_PSET: the union of all Korobov lattice point sets of
 * Section 2.2 for a prime K (= N of the descriptor): the (K-1)^2 points
 * n·(1, γ, γ^2, ..., γ^{s-1}) / K mod 1, n, γ = 1..K-1.  gen_host is ignored
 * (may be NULL), row0 must be AUTO or EXCLUDE (the set has no zero point),
 * prec FP32.  Output rows: (γ-1)(K-1) + (n-1) in conventional order, or
 * block b, row r of the reordered blocks Y'_{b+1} = Z·P_{b+1} (γ = g^b,
 * n = g^{-r}) in circulant order.  Every block shares one circulant Z, so
 * the K-1 products run as one product with (K-1)·t right-hand sides.
 * qmc_matmul (without row_mean / exp_sum) and qmc_generate_points accept
 * p-set plans; the adjoint, batch and no-allocation calls return
 * QMC_ERR_UNSUPPORTED. */
/* QMC_LATTICE_FB: a polynomial lattice rule over F_b for a prime base b
 * (Remark 1: the method carries over to polynomial lattice rules over a
 * finite field).  N = b^m, the modulus P(x) is a monic primitive polynomial
 * of degree m over F_b, named by its base-b encoding Σ_i p_i b^i (so
 * b^m <= modulus_P < 2 b^m for the leading coefficient 1; 0 = the smallest
 * primitive one), and q_j(x) by the encoding Σ_i c_i b^i in [1, N-1].  Point
 * n (base-b digits n_i, n(x) = Σ n_i x^i) has coordinates
 * v_m(n(x) q_j(x) mod P / P) with v_m(Σ_k u_k x^{-k}) = Σ_{k<=m} u_k b^{-k}.
 * With x primitive, q_j = x^{e_j}, the reordering and the circulant are
 * those of the F_2 kind with L = b^m - 1.  b = 2 gives the F_2 kind's
 * points and tables. */
typedef enum { QMC_LATTICE_PRIME = 0, QMC_LATTICE_F2 = 1, QMC_KOROBOV_PSET = 2, QMC_LATTICE_FB = 3 } qmc_kind;

/* Coordinate maps φ of Section 2.1 (identity, Φ^{-1}, tent) and the
 * centred map x - 1/2 used by the uniform-coefficient experiment
 * (Section 4, Experiment 2). */
typedef enum {
  QMC_MAP_IDENTITY = 0,
  QMC_MAP_CENTRED = 1,
  QMC_MAP_PHI_INV = 2,
  QMC_MAP_TENT = 3
} qmc_map;

/* Row 0 (the point x_0 = 0, Section 2.1): AUTO keeps it iff φ(0) is finite
 * (dropped for Φ^{-1}, where φ(0) = -inf). */
typedef enum { QMC_ROW0_AUTO = 0, QMC_ROW0_INCLUDE = 1, QMC_ROW0_EXCLUDE = 2 } qmc_row0;

/* Output row order.  CONVENTIONAL: row n holds y_n·A with
 * x_n = ({n z_j / N})_j (F_2: n read as the bit polynomial n(x)).
 * CIRCULANT: the reordered order of Section 2.1 (row r+1 holds the point
 * g^{-r}), which skips the un-permute gather. */
typedef enum { QMC_ORDER_CONVENTIONAL = 0, QMC_ORDER_CIRCULANT = 1 } qmc_order;

/* Arithmetic of the product.  FP32: columns of A are paired as (re, im) of
 * one complex FFT column.  FP32_SPLIT (FP64 A only): each column is split
 * into hi = fp32(a) and lo = fp32(a - hi), carried as (re, im), and the
 * result is re + im, which removes the input rounding of A. */
typedef enum { QMC_PREC_FP32 = 0, QMC_PREC_FP32_SPLIT = 1 } qmc_prec;

typedef enum { QMC_DTYPE_F32 = 0, QMC_DTYPE_F64 = 1 } qmc_dtype;

typedef struct {
  int32_t kind;          /* qmc_kind */
  int64_t N;             /* prime N (< 2^31), 2^m with 2 <= m <= 30, or b^m < 2^31 (F_b, N >= 4) */
  uint64_t modulus_P;    /* F_2: bit i = coefficient of x^i, degree m; F_b: Σ_i p_i b^i;
                            0 = the smallest primitive one */
  int64_t g;             /* prime only: primitive root; 0 = smallest primitive root */
  int32_t s;             /* number of coordinates (rows of A), >= 1 */
  const int64_t* gen_host; /* s entries: z_j in [1, N-1] (prime) or q_j bit polynomial (F_2),
                              or e_j in [0, L-1] when gen_is_exponent = 1 */
  int32_t gen_is_exponent;
  int32_t map;           /* qmc_map */
  int32_t row0;          /* qmc_row0 */
  int32_t order;         /* qmc_order */
  int32_t prec;          /* qmc_prec */
  double shift;          /* diagonal shift Δ in [0, 1) (Remark 2): every coordinate x of every
                            point becomes {x + Δ} before φ, so z_k = φ({x_k + Δ}) and row 0 is
                            φ(Δ)·Σ_j a_j; 0 = unshifted.  The same Δ in every coordinate keeps
                            Y' = Z·P; a different shift per coordinate would not (not offered). */
  int32_t base;          /* F_b only: the prime b (2 <= b < 256); ignored by the other kinds */
} qmc_desc;

typedef struct {
  int64_t N;
  int64_t L;             /* circulant size: N-1 (prime) or 2^m - 1 (F_2) */
  int64_t g;             /* primitive root used (prime) */
  uint64_t modulus_P;    /* modulus used (F_2) */
  int32_t s;
  int32_t n_distinct;    /* number of distinct e_j (nonzero rows of P·A) */
  int32_t collision_adds;/* s - n_distinct: additions spent by the scatter-add */
  int32_t row0_adds;     /* additions for y_0·a: s-1 when row 0 is kept and φ(0) != 0, else 0 */
  int64_t out_rows;      /* N or N-1 */
  double phi0;           /* φ at the row-0 point: φ(0), or φ(Δ) with a diagonal shift */
  int32_t L1, L2;        /* FFT factorisation L = L1·L2 (L2 = 1: single pass) */
  int32_t has_row0;
  int32_t base;          /* field size b of a polynomial lattice (2 for F_2), 0 for prime N */
} qmc_info;

/* Tables a plan can copy back for bit-exact checks (qmc_plan_copy_table). */
typedef enum {
  QMC_TABLE_POW = 0,       /* int32[L]: g^k mod N, or x^k mod P as an integer (base-b encoding) */
  QMC_TABLE_LOG = 1,       /* int32[N]: discrete log, -1 at 0 */
  QMC_TABLE_EXPONENTS = 2, /* int32[s]: e_j */
  QMC_TABLE_OUT_ROW = 3,   /* int32[L]: output row of circulant row r */
  QMC_TABLE_ZETA = 4,      /* double[L]: generator sequence z_k = φ(point of g^k) */
  QMC_TABLE_SPECTRUM64 = 5,/* double[2L]: conj(DFT(z))/L in the FFT's internal order */
  QMC_TABLE_ROW_PTR = 6,   /* int32[L+1]: CSR offsets of positions into the j list */
  QMC_TABLE_JLIST = 7      /* int32[s]: j sorted by (e_j, j) */
} qmc_table;

/* Builds every plan table on the device: powers and discrete logs of g (or
 * of x mod P), the exponents e_j, the position -> j lists used by the
 * scatter-add, the output-row permutation, the generator sequence z_k in
 * FP64 and its spectrum in FP64 (stored as FP32 for the product and FP64
 * for checks), and FP64-derived twiddles.  Section 2.1 (the setup before
 * Eq. (3)).  Synchronous on `stream`.  On error *plan is set to NULL. */
int qmc_plan_create(void** plan, const qmc_desc* desc, void* stream);

int qmc_plan_destroy(void* plan);

/* Plain facts about the plan (host struct, filled synchronously). */
int qmc_plan_info(void* plan, qmc_info* info_host);

/* Section 2.1 (end): storing beta and c_1..c_s suffices to regenerate Y.
 * Writes the s exponents e_j = c_j - 1 (host int32 array). */
int qmc_plan_exponents(void* plan, int32_t* e_host);

/* Copies a plan table to host memory (bytes must equal the table size).
 * Synchronous. */
int qmc_plan_copy_table(void* plan, int32_t which, void* dst_host, int64_t bytes);

/* Ensures plan-owned scratch for products with up to t columns, so that
 * later calls (and CUDA-graph capture of them) do not allocate. */
int qmc_plan_reserve(void* plan, int32_t t_max);

/* Reads and clears the plan's device error word; synchronises `stream`.
 * Libraries compiled with -DQMC_CHECK_BOUNDS (libqmcfft_checked.so) check
 * every index their kernels read from a plan table against the buffer it
 * addresses; a failed check latches QMC_ERR_BOUNDS here instead of
 * trapping (see qmc_debug.h for the test hook of those builds).  The
 * default build compiles the checks out. */
int qmc_plan_sync_status(void* plan, void* stream);

/* B = Y·A (Section 2.1, Eq. (3), plus y_0·a for row 0).
 *   A        device, s x t, row-major, leading dimension lda >= t,
 *            element type a_dtype (QMC_DTYPE_F32 or F64; FP32_SPLIT needs F64)
 *   out      device float, out_rows x t, leading dimension ldo >= t
 *   row_mean nullable device float[out_rows]: (1/t) Σ_k B_nk
 *   exp_sum  nullable device double[1]: Σ_{n,k} exp(B_nk) (overwritten)
 * Allocates plan scratch on first use for a given t (see qmc_plan_reserve).
 * The un-permute pass writes each output row in pieces of 64 or 128 bytes;
 * when t is odd, choosing ldo so that the row stride is a multiple of 32
 * bytes avoids pieces that straddle 32-byte sectors (measured on N = 786433,
 * t = 4225: 8.7 ms for that pass at ldo = t, 7.4 ms at ldo = 4232). */
int qmc_matmul(void* plan, const void* A, int64_t lda, int32_t t, int32_t a_dtype,
               float* out, int64_t ldo, float* row_mean, double* exp_sum, void* stream);

/* The paper has no counterpart to this entry point.  It computes the same
 * B = Y·A as qmc_matmul (no row_mean / exp_sum epilogues) but allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.  It is
 * for callers that must not allocate device memory while they run, for
 * example a serving loop that owns a fixed memory budget or a caller whose
 * allocator cannot be entered at that point.  (The plan itself is built
 * beforehand by qmc_plan_create, which does allocate.)
 *
 * The scratch it needs (column statistics and, when L > 1024, the L x T
 * work array between the FFT passes) lives in one fixed 32 MiB device array
 * inside the library, which every GPU that loads the library holds until the
 * process exits.  A problem that needs more than 32 MiB of scratch is
 * rejected with QMC_ERR_SCRATCH before any work is launched (a prime plan
 * with L = 65536 and FP32 input takes t up to 112; plans with L <= 1024
 * need only the statistics, a few bytes per column).
 *
 * The first call on each device looks up that array's device address with
 * the device current and keeps it; make that first call before any stream
 * capture.  The kept address belongs to the device's primary context: after
 * cudaDeviceReset on a device, do not call this entry point on that device
 * again in the same process.  Every call shares the one array: two calls
 * whose kernels overlap on the GPU (different streams or host threads) race
 * on it and must be ordered by the caller.  Arguments and errors are those
 * of qmc_matmul, except that Korobov p-set plans (QMC_KOROBOV_PSET) return
 * QMC_ERR_UNSUPPORTED. */
int qmc_matmul_noalloc(void* plan, const void* A, int64_t lda, int32_t t, int32_t a_dtype,
                       float* out, int64_t ldo, void* stream);

/* B = exp?(c + Y·A): the product with an affine output map, the form the
 * paper's applications take.  Section 3.2 (uniform coefficients) assembles
 * b_{k,l} = a_{0,k,l}·1 + Y·a_{k,l} (a column offset, apply_exp = 0);
 * Section 3.3 (log-normal coefficients) forms Θ = Ψ̂ + Y·Ψ and needs
 * a = exp(Θ) (column offset and apply_exp = 1).  Out element (n, k) is
 * col_offset[k] + (Y·A)_nk, then exp() when apply_exp = 1; row 0, when
 * kept, gets the same map.
 *   col_offset  device float[t], or NULL for no offset
 *   apply_exp   0 or 1 (anything else: QMC_ERR_INVALID)
 * Other arguments, layouts and errors as qmc_matmul (no row mean or exp
 * sum here).  Korobov p-set plans apply the map to every block. */
int qmc_matmul_affine(void* plan, const void* A, int64_t lda, int32_t t, int32_t a_dtype,
                      const float* col_offset, int32_t apply_exp, float* out, int64_t ldo, void* stream);

/* dA = Yᵀ·G, the adjoint of qmc_matmul: the transposed circulant applied
 * with the conjugate spectrum, gathered back to the s rows e_j (colliding j
 * receive the same row), plus φ(0)·G_0 for row 0 when kept.
 *   G        device float, out_rows x t, leading dimension ldg
 *   g_mode   0: G is the cotangent dL/dB.
 *            1: G holds B and the cotangent is exp(B)/(out_rows·t), the
 *               gradient of L = mean exp(B) (fused, nothing materialised).
 *   dA       device float, s x t, leading dimension ldda (overwritten) */
int qmc_matmul_backward(void* plan, const float* G, int64_t ldg, int32_t t, int32_t g_mode,
                        float* dA, int64_t ldda, void* stream);

/* Materialises Y (out_rows x s, FP32, row-major, leading dimension ldy),
 * in the plan's output order, for the dense-GEMM comparison (Section 4,
 * Experiment 1's standard approach) and for Section 2.1's remark that
 * Eq. (3) also generates the points quickly. */
int qmc_generate_points(void* plan, float* Y, int64_t ldy, void* stream);

/* The finite-element step that follows the product in Sections 3.2 and 3.3
 * (Experiments 2 and 3): hat functions φ_k at x_k = k/M on (0, 1) with zero
 * boundary values give, for each point y_n, a symmetric tridiagonal
 * stiffness matrix B(y_n) of size M-1; the step solves B(y_n) û^(n) = ĝ for
 * every n and writes the estimate ū = (1/n_sys) Σ_n û^(n) of the expected
 * finite-element coefficients (Section 3.2's average over the QMC points).
 *   B       device float, n_sys rows, leading dimension ldb floats; row n
 *           holds point y_n's stiffness data, by kind:
 *           QMC_FE_TRIDIAG: the M-1 diagonal entries b_{k,k}, k = 1..M-1,
 *             then the M-2 entries b_{k,k+1}, k = 1..M-2 (2M-3 floats: the
 *             columns a_0 + Y·a_{k,l} of Section 3.2, qmc_matmul_affine);
 *           QMC_FE_MIDPOINT: the coefficient a(x_i, y_n) at the M element
 *             midpoints x_i = (i - 1/2)/M (M floats: Section 3.3's exp(Θ),
 *             qmc_matmul_affine with apply_exp), assembled with one
 *             equal-weight point per element: b_{k,k} = M (a_k + a_{k+1}),
 *             b_{k,k+1} = -M a_{k+1}.
 *   g_hat   nullable device double[M-1]: ĝ_k = ∫ g φ_k (NULL: all ones,
 *           as in the experiments).
 *   work    device scratch of qmc_fe_work_bytes(n_sys, M) bytes, 8-byte
 *           aligned, owned by the caller; contents need not be initialised.
 *   u_mean  device double[M-1], overwritten with ū.
 * QMC_FE_TRIDIAG: for M <= 8192 each system is first solved by defect
 * correction: the rows' off-diagonals define an element-difference matrix
 * K_f (the midpoint form's structure), the rest of the diagonal is
 * δ = diag - diag(K_f), and u <- K_f^{-1}(ĝ - δ ⊙ u) is iterated (K_f^{-1}
 * by prefix sums, first in FP32, then in pairs of FP32 numbers) until the
 * estimated error is below 2^-40 of the solution; Experiment 2's rows,
 * whose δ is their FP32 rounding, settle in a few steps.  A system that
 * does not settle, or any system when M > 8192, is solved by a block of
 * 128 threads in FP64: the unknowns are cut into chunks, each chunk
 * eliminated without pivoting to give its response to the values at the
 * chunk boundaries, the boundary (interface) values solved from their own
 * tridiagonal system, and every chunk back-substituted; each system is
 * first scaled by a power of two, which keeps the pivots inside the range
 * of the FP32 starting value of their reciprocals.  It assumes positive
 * definite matrices (as the experiments' are) and does not check for zero
 * pivots.  The mean sums the systems in index order.
 * QMC_FE_MIDPOINT: the matrix is the element-difference form
 * Dᵀ diag(M a) D, whose solution follows from prefix sums of the element
 * fluxes: with r_i = 1/a_i and G_j = ĝ_1 + ... + ĝ_j,
 * û_k = (1/M) Σ_{i<=k} (q_1 - G_{i-1}) r_i, q_1 = Σ_i G_{i-1} r_i / Σ_i r_i,
 * so the mean needs two sums along each row, two column sums over the
 * systems and one prefix sum (no elimination).  The row and column sums
 * run in pairs of FP32 numbers (about 47 significant bits), the rest in
 * FP64; each system and ĝ's prefix sums are scaled by powers of two.  It
 * assumes a_i > 0 with each system's coefficients within a factor 2^100 of
 * one another.
 * Both forms add the same data in the same order on every call
 * (deterministic).  Asynchronous on stream.  QMC_ERR_INVALID: null B, work
 * or u_mean, M < 3, n_sys < 1, a bad kind, misaligned work; QMC_ERR_SHAPE:
 * ldb below the row length, work_bytes below the need, or (midpoint) more
 * than 2^31 - 1 column-sum blocks; QMC_ERR_CUDA: a failed launch.  Nothing
 * touches the device before the arguments pass these checks. */
typedef enum { QMC_FE_TRIDIAG = 0, QMC_FE_MIDPOINT = 1 } qmc_fe_kind;
int64_t qmc_fe_work_bytes(int64_t n_sys, int32_t M);
int qmc_fe_solve_mean(const float* B, int64_t ldb, int64_t n_sys, int32_t M, int32_t kind,
                      const double* g_hat, void* work, int64_t work_bytes, double* u_mean, void* stream);

/* Batched forward products B_i = Y_i·A_i over many plans (uneven N, s, t;
 * FP32 A), an extension of Section 1's product to many instances.
 *   qmc_batch_create   plans and their column counts t (host arrays of
 *                      `count`); reserves each plan's scratch.  The batch
 *                      keeps pointers to the plans, which must outlive it.
 *   qmc_batch_matmul   A_i, lda_i, out_i, ldo_i: host arrays of `count`
 *                      entries holding device pointers / leading dims.
 * Modes (qmc_batch_set_option, QMC_BATCH_OPT_MODE):
 *   QMC_BATCH_GRAPH (default): the first call autotunes (per-problem pass
 *     kernel, number of concurrent branches) and captures all products
 *     into one CUDA graph; later calls with the same pointers are one graph
 *     launch; new pointers re-capture.  The first call runs each product
 *     several times while tuning (outputs end up correct).
 *   QMC_BATCH_PERSISTENT: the column statistics of all problems (two
 *     launches), then one persistent launch drains a stage-major
 *     (problem, pass, chunk of tiles) queue; a chunk waits, with a bounded
 *     wait, for the previous pass of its problem.  The passes of the
 *     768 x 1024 transform (and its sparse first pass) run the tile loops
 *     of their specialised persistent kernels, passes of length 256 the
 *     register tile, every other pass the generic shared-memory tile.  The
 *     queue's description is uploaded only when the problems or pointers
 *     change.  A wait that exceeds QMC_BATCH_OPT_WAIT_LIMIT_US latches
 *     QMC_ERR_TIMEOUT, read by qmc_batch_sync_status, and every block of
 *     the launch returns. */
typedef enum { QMC_BATCH_GRAPH = 0, QMC_BATCH_PERSISTENT = 1 } qmc_batch_mode;
typedef enum {
  QMC_BATCH_OPT_MODE = 0,           /* qmc_batch_mode */
  QMC_BATCH_OPT_BRANCHES = 1,       /* graph branches, 0 = autotune (default), up to 16 */
  QMC_BATCH_OPT_WAIT_LIMIT_US = 2,  /* bounded wait of the persistent mode (default 1 s) */
  QMC_BATCH_OPT_TEST_BLOCK_ITEM = 3 /* test hook: the dependency of this work item (index in
                                       pass-major order) is made unreachable */
} qmc_batch_option;

int qmc_batch_create(void** batch, void* const* plans, const int32_t* t_host, int32_t count,
                     void* stream);
int qmc_batch_set_option(void* batch, int32_t option, int64_t value);
int qmc_batch_matmul(void* batch, const float* const* A_host_ptrs, const int64_t* lda_host,
                     float* const* out_host_ptrs, const int64_t* ldo_host, void* stream);
/* Reads and clears the batch's device error word; synchronises `stream`. */
int qmc_batch_sync_status(void* batch, void* stream);
int qmc_batch_destroy(void* batch);

/* Kernel stages, for the per-stage timing of qmc_plan_read_profile(). */
typedef enum {
  QMC_STAGE_ROW0 = 0,          /* column sums and scales; y_0·A = φ(0)·colsum(A) */
  QMC_STAGE_FWD_SCATTER = 1,   /* scatter-add + forward FFT over n1 + twiddle */
  QMC_STAGE_FWD_SPECTRAL = 2,  /* forward FFT over n2, ×H, inverse FFT, twiddle */
  QMC_STAGE_FWD_UNPERMUTE = 3, /* inverse FFT over k1 + un-permute (+ epilogues) */
  QMC_STAGE_FWD_FUSED = 4,     /* single-pass product (L <= 1024) */
  QMC_STAGE_BWD_GATHER = 5,    /* adjoint: permuted gather of G + forward FFT over n1 */
  QMC_STAGE_BWD_SPECTRAL = 6,  /* adjoint: ×conj(H) */
  QMC_STAGE_BWD_SCATTER = 7,   /* adjoint: inverse FFT + write rows e_j of dA */
  QMC_STAGE_BWD_FUSED = 8,     /* single-pass adjoint */
  QMC_STAGE_BATCH = 9,         /* persistent batched launch */
  QMC_STAGE_ROW_MEAN = 10,     /* row mean by linearity: row averages of A and their product */
  QMC_STAGE_DENSE_SCATTER = 11,/* P·A streamed into the work array (densely hit positions) */
  QMC_STAGE_SPARSE_PACK = 12,  /* sparse first pass: A's rows packed by 8-column panel */
  QMC_STAGE_FWD_SPARSE = 13,   /* sparse first pass: spectral pass summing its lines from A */
  QMC_NUM_STAGES = 14
} qmc_stage;

/* Plan options (qmc_plan_set_option). */
typedef enum {
  QMC_OPT_PASS_KERNEL = 0,  /* qmc_pass_kernel: which FFT pass kernel products use */
  QMC_OPT_ROW_MEAN = 1,     /* qmc_row_mean_mode: how qmc_matmul forms row_mean */
  QMC_OPT_FIRST_PASS = 2,   /* qmc_first_pass: how a forward product forms its first pass */
  QMC_OPT_FFT_SPLIT = 3     /* L1 of the transform's factorisation L = L1·L2 (see below) */
} qmc_option;

/* QMC_OPT_FFT_SPLIT: re-factors the circulant's transform as L = L1·L2 with
 * the given L1 (L2 = L / L1; L1 = L for a single pass; 0 = the library's
 * default: a single pass when L <= 1024, else the split with the shortest
 * longer factor) and rebuilds every table that depends on the split (line
 * buckets, gather and entry lists, the spectrum in the transform's order).
 * Both factors must be at most 1024 and products of the supported radices.
 * Results agree with any other split to FP32 rounding.  Synchronous: it
 * waits for the device, so call it when no product of this plan is in
 * flight.  QMC_ERR_INVALID: L1 does not divide L or a factor exceeds 1024;
 * QMC_ERR_UNSUPPORTED: a factor has an unsupported prime or the plan is a
 * Korobov p-set (whose blocks fix the first pass).  After an error the plan
 * keeps its previous split. */

/* First FFT pass of a two-pass forward product (L = L1·L2, Section 2.1's
 * scatter-add P·A followed by the transform).  TRANSFORM scatters A's rows
 * into the L x T work array and transforms each length-L1 line.  SPARSE
 * skips that pass: the spectral pass forms each of its lines directly from
 * the rows of A, as Σ_j a_j·w_L^{-e_j·k1} over the rows whose position e_j
 * falls on the line (pass length L2 = 256 or 1024, at least 8 complex columns,
 * QMC_KERNEL_AUTO or PIPELINED; otherwise TRANSFORM runs).  Its cost grows
 * with s·L1 instead of L, so AUTO takes it when s <= L2. */
typedef enum { QMC_FIRST_PASS_AUTO = 0, QMC_FIRST_PASS_TRANSFORM = 1, QMC_FIRST_PASS_SPARSE = 2 } qmc_first_pass;

/* Per-row mean r_n = (1/t) Σ_k B_nk of qmc_matmul.  LINEAR (default) uses
 * r = Y·(A·1/t): one more single-column product after the main one.  FUSED
 * adds each output tile's row sums into r with one atomic per row and tile
 * inside the un-permute pass (result order-dependent in the last bits). */
typedef enum { QMC_ROW_MEAN_LINEAR = 0, QMC_ROW_MEAN_FUSED = 1 } qmc_row_mean_mode;

typedef enum {
  QMC_KERNEL_AUTO = 0,      /* fastest available: PIPELINED, then REGISTER, then GENERIC */
  QMC_KERNEL_GENERIC = 1,   /* shared-memory Stockham kernel for every pass */
  QMC_KERNEL_REGISTER = 2,  /* register-resident kernel (pass lengths 256, 1024), else GENERIC */
  QMC_KERNEL_PIPELINED = 3  /* persistent double-buffered register kernel for the work-array
                               passes (pass lengths 256, 1024, 8-column panels), else REGISTER */
} qmc_pass_kernel;

/* Sets a plan option; QMC_ERR_INVALID for an unknown option or value. */
int qmc_plan_set_option(void* plan, int32_t option, int64_t value);

/* When enabled, every later product on this plan brackets each kernel it
 * launches with CUDA events on the launching stream.  Off by default. */
int qmc_plan_set_profiling(void* plan, int32_t enable);

/* Synchronises the recorded events, writes per-stage totals (milliseconds,
 * host double[QMC_NUM_STAGES]) and launch counts (host int32[QMC_NUM_STAGES]),
 * and clears the record. */
int qmc_plan_read_profile(void* plan, double* ms_host, int32_t* launches_host);

/* Number of kernels the library has launched on the product paths (row 0,
 * passes, batch) since it was loaded. */
int64_t qmc_kernel_launches(void);

const char* qmc_status_string(int status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int qmc_version(void);

#ifdef __cplusplus
}
#endif

#endif  /* QMC_H_ */
