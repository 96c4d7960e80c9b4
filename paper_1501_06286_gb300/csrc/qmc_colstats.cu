// qmc_colstats.cu — per-column statistics of the product's input, computed
// before the FFT passes:
//   * sum_k = Σ_j A_jk, from which row 0 is y_0·a = φ(0)·Σ_j a_j
//     (Section 2.1), accumulated in FP64;
//   * l1_k = Σ_j |A_jk|, from which a power-of-two column scale is taken.
//
// Two real columns travel as the real and imaginary part of one complex
// FFT column.  Rounding inside the complex transform mixes the two parts,
// so each output column carries an error proportional to the larger of the
// pair.  Scaling every column by 2^-e with 2^e <= l1_k < 2^(e+1) before the
// transform (and by 2^e after) equalises the pair without adding any
// rounding, and an all-zero column gets scale 0 so that it comes out as
// exact zeros.
#include <math.h>

#include "qmc_internal.h"

namespace qmc {

// Rows per partial-sum chunk: a multiple of 64, and at most 16 chunks.
static int stat_chunk_rows(int rows) {
  int c = (rows + 15) / 16;
  c = ((c + 63) / 64) * 64;
  return c < 64 ? 64 : c;
}

// Stage 1: partial sums over a chunk of rows for 32 columns per block;
// each thread reads 8 rows per step so that 8 loads are in flight.
// Block (bx, chunk) of the (32, 8) thread grid.
__device__ __forceinline__ void colstats_partial_tile(const void* X, int64_t ldx, int rows, int t, int x_f64,
                                                      int x_exp, float x_scale, int chunk_rows, double* part_sum,
                                                      double* part_l1, int bx, int chunk) {
  __shared__ double ssum[8][33], sl1[8][33];
  const int k = bx * 32 + threadIdx.x;
  const int r0 = chunk * chunk_rows, r1 = min(rows, r0 + chunk_rows);
  double sum = 0.0, l1 = 0.0;
  if (k < t && x_f64) {
    for (int rb = r0 + threadIdx.y; rb < r1; rb += 64) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = rb + 8 * q;
        v[q] = r < r1 ? reinterpret_cast<const double*>(X)[(int64_t)r * ldx + k] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) { sum += v[q]; l1 += fabs(v[q]); }
    }
  } else if (k < t) {
    // FP32 input: compensated (Kahan) FP32 sum, plain FP32 l1 (only its
    // binary exponent is used); GB300's FP64 rate is a small fraction of FP32.
    float s = 0.f, comp = 0.f, a1 = 0.f;
    for (int rb = r0 + threadIdx.y; rb < r1; rb += 64) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = rb + 8 * q;
        v[q] = r < r1 ? reinterpret_cast<const float*>(X)[(int64_t)r * ldx + k] : 0.f;
        if (x_exp && r < r1) v[q] = expf(v[q]) * x_scale;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float y = v[q] - comp;
        const float tt = s + y;
        comp = (tt - s) - y;
        s = tt;
        a1 += fabsf(v[q]);
      }
    }
    sum = (double)s - (double)comp;
    l1 = (double)a1;
  }
  ssum[threadIdx.y][threadIdx.x] = sum;
  sl1[threadIdx.y][threadIdx.x] = l1;
  __syncthreads();
  if (threadIdx.y == 0 && k < t) {
    double s = 0.0, a = 0.0;
    for (int y = 0; y < 8; ++y) { s += ssum[y][threadIdx.x]; a += sl1[y][threadIdx.x]; }
    part_sum[(int64_t)chunk * t + k] = s;
    part_l1[(int64_t)chunk * t + k] = a;
  }
}

__global__ void k_colstats_partial(const void* X, int64_t ldx, int rows, int t, int x_f64, int x_exp,
                                   float x_scale, int chunk_rows, double* part_sum, double* part_l1) {
  colstats_partial_tile(X, ldx, rows, t, x_f64, x_exp, x_scale, chunk_rows, part_sum, part_l1, (int)blockIdx.x,
                        (int)blockIdx.y);
}

// Stage 2: fixed-order reduction over chunks (warp y of a block sums the
// chunks y, y+8, ... of 32 columns; the 8 warp sums are added in order);
// writes the column scales and, for the forward product with row 0 kept,
// row 0 and its epilogue terms.
__device__ __forceinline__ void colstats_final_tile(const double* part_sum, const double* part_l1, int chunks,
                                                    int t, float* scale, float* inv, double phi0, float* out_row0,
                                                    float* row_mean0, float inv_t, double* exp_sum, int* err,
                                                    int bx) {
  __shared__ double ssum[8][33], sl1[8][33];
  const int k = bx * 32 + threadIdx.x;
  {
    double s = 0.0, a = 0.0;
    if (k < t) {
      for (int c = threadIdx.y; c < chunks; c += 8) {
        s += part_sum[(int64_t)c * t + k];
        a += part_l1[(int64_t)c * t + k];
      }
    }
    ssum[threadIdx.y][threadIdx.x] = s;
    sl1[threadIdx.y][threadIdx.x] = a;
  }
  __syncthreads();
  if (threadIdx.y != 0) return;
  float b0 = 0.f;
  if (k < t) {
    double s = 0.0, a = 0.0;
    for (int y = 0; y < 8; ++y) { s += ssum[y][threadIdx.x]; a += sl1[y][threadIdx.x]; }
    // a NaN or infinity anywhere in the column: the plan's error word
    // records it (the outputs of the column and of its complex partner are
    // not finite)
    if (err && !(isfinite(a) && isfinite(s))) atomicOr(err, kErrNonFinite);
    if (a > 0.0 && isfinite(a)) {
      int e = ilogb(a);
      e = max(-100, min(100, e));
      scale[k] = (float)ldexp(1.0, -e);
      inv[k] = (float)ldexp(1.0, e);
    } else {
      scale[k] = 0.f;
      inv[k] = 0.f;
    }
    if (out_row0) {
      b0 = (float)(phi0 * s);
      out_row0[k] = b0;
      if (exp_sum) atomicAdd(exp_sum, exp((double)b0));
    }
  }
  if (out_row0 && row_mean0) {
    for (int off = 16; off > 0; off >>= 1) b0 += __shfl_xor_sync(0xffffffffu, b0, off);
    if (threadIdx.x == 0) atomicAdd(row_mean0, b0 * inv_t);
  }
}

__global__ void k_colstats_final(const double* part_sum, const double* part_l1, int chunks, int t,
                                 float* scale, float* inv, double phi0, float* out_row0,
                                 float* row_mean0, float inv_t, double* exp_sum, int* err) {
  colstats_final_tile(part_sum, part_l1, chunks, t, scale, inv, phi0, out_row0, row_mean0, inv_t, exp_sum, err,
                      (int)blockIdx.x);
}

// Many problems in one launch per stage (the batch's persistent mode): a
// block finds its job from the jobs' first block numbers.
__device__ __forceinline__ int job_of(const ColstatsJob* jobs, int njobs, int final_stage) {
  int lo = 0, hi = njobs - 1;
  const int b = (int)blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((final_stage ? jobs[mid].blk_final : jobs[mid].blk_partial) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_colstats_partial_multi(const ColstatsJob* __restrict__ jobs, int njobs) {
  const ColstatsJob& j = jobs[job_of(jobs, njobs, 0)];
  const int local = (int)blockIdx.x - j.blk_partial, gx = (j.t + 31) / 32;
  colstats_partial_tile(j.X, j.ldx, j.rows, j.t, 0, 0, 1.f, j.chunk_rows, j.part_sum, j.part_l1, local % gx,
                        local / gx);
}

__global__ void k_colstats_final_multi(const ColstatsJob* __restrict__ jobs, int njobs) {
  const ColstatsJob& j = jobs[job_of(jobs, njobs, 1)];
  colstats_final_tile(j.part_sum, j.part_l1, j.chunks, j.t, j.scale, j.inv, j.phi0, j.out_row0, nullptr,
                      1.0f / (float)j.t, nullptr, j.err, (int)blockIdx.x - j.blk_final);
}

void colstats_job(void* work, const float* X, int64_t ldx, int rows, int t, double phi0, float* out_row0,
                  int* err, ColstatsJob* job, float** scale_out, float** inv_out) {
  const int chunk_rows = stat_chunk_rows(rows);
  const int chunks = (rows + chunk_rows - 1) / chunk_rows;
  ColstatsJob& j = *job;
  j = ColstatsJob{};
  j.X = X; j.ldx = ldx; j.rows = rows; j.t = t; j.chunk_rows = chunk_rows; j.chunks = chunks;
  j.part_sum = reinterpret_cast<double*>(work);
  j.part_l1 = j.part_sum + (size_t)chunks * t;
  j.scale = reinterpret_cast<float*>(j.part_l1 + (size_t)chunks * t);
  j.inv = j.scale + t;
  j.phi0 = phi0; j.out_row0 = out_row0; j.err = err;
  j.blocks_partial = ((t + 31) / 32) * chunks;
  j.blocks_final = (t + 31) / 32;
  *scale_out = j.scale;
  *inv_out = j.inv;
}

int launch_colstats_multi(const ColstatsJob* jobs, int njobs, int partial_blocks, int final_blocks,
                          cudaStream_t st) {
  if (njobs < 1) return QMC_OK;
  k_colstats_partial_multi<<<partial_blocks, dim3(32, 8), 0, st>>>(jobs, njobs);
  count_launch();
  k_colstats_final_multi<<<final_blocks, dim3(32, 8), 0, st>>>(jobs, njobs);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

size_t colstats_bytes(int rows, int t) {
  const int chunks = (rows + stat_chunk_rows(rows) - 1) / stat_chunk_rows(rows);
  return (size_t)chunks * t * 2 * sizeof(double) + (size_t)t * 2 * sizeof(float);
}

int launch_colstats(void* work, const void* X, int64_t ldx, int rows, int t, int x_f64, int x_exp,
                    float x_scale, double phi0, float* out_row0, float* row_mean0, double* exp_sum,
                    float** scale_out, float** inv_out, cudaStream_t st, int* err) {
  const int chunk_rows = stat_chunk_rows(rows);
  const int chunks = (rows + chunk_rows - 1) / chunk_rows;
  double* part_sum = reinterpret_cast<double*>(work);
  double* part_l1 = part_sum + (size_t)chunks * t;
  float* scale = reinterpret_cast<float*>(part_l1 + (size_t)chunks * t);
  float* inv = scale + t;
  dim3 g1((t + 31) / 32, chunks), b1(32, 8);
  k_colstats_partial<<<g1, b1, 0, st>>>(X, ldx, rows, t, x_f64, x_exp, x_scale, chunk_rows, part_sum,
                                        part_l1);
  count_launch();
  k_colstats_final<<<(t + 31) / 32, b1, 0, st>>>(part_sum, part_l1, chunks, t, scale, inv, phi0,
                                                 out_row0, row_mean0, 1.0f / (float)t, exp_sum, err);
  count_launch();
  *scale_out = scale;
  *inv_out = inv;
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // namespace qmc

namespace qmc {

// abar_j = (1/t) Σ_k A_jk (one warp per row; FP64 accumulation for FP64
// input, compensated FP32 otherwise), stored in A's element type.
__global__ void k_row_average(const void* A, int64_t lda, int s, int t, int a_f64, void* abar) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= s) return;
  if (a_f64) {
    const double* row = reinterpret_cast<const double*>(A) + (int64_t)warp * lda;
    double acc = 0.0;
    for (int k = lane; k < t; k += 32) acc += row[k];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) reinterpret_cast<double*>(abar)[warp] = acc / (double)t;
  } else {
    const float* row = reinterpret_cast<const float*>(A) + (int64_t)warp * lda;
    float acc = 0.f, comp = 0.f;
    for (int k = lane; k < t; k += 32) {
      const float y = row[k] - comp;
      const float tt = acc + y;
      comp = (tt - acc) - y;
      acc = tt;
    }
    double d = (double)acc - (double)comp;
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (lane == 0) reinterpret_cast<float*>(abar)[warp] = (float)(d / (double)t);
  }
}

int launch_row_average(const void* A, int64_t lda, int s, int t, int a_f64, void* abar, cudaStream_t st) {
  const int nt = 256;
  const int blocks = (int)(((int64_t)s * 32 + nt - 1) / nt);
  k_row_average<<<blocks, nt, 0, st>>>(A, lda, s, t, a_f64, abar);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

// Row 0 of qmc_matmul_affine: out[k] = col_off[k] + out[k], then exp().
__global__ void k_row0_affine(float* out_row0, int t, const float* col_off, int out_exp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < t) {
    float b = out_row0[k];
    if (col_off) b += col_off[k];
    out_row0[k] = out_exp ? expf(b) : b;
  }
}

int launch_row0_affine(float* out_row0, int t, const float* col_off, int out_exp, cudaStream_t st) {
  k_row0_affine<<<(t + 255) / 256, 256, 0, st>>>(out_row0, t, col_off, out_exp);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // namespace qmc

namespace qmc {

// Scatter-add a' = P·A (Section 2.1) as a streaming pass, for plans whose
// positions are densely hit (s comparable to L or larger, the regime of the
// applications of Sections 3.2 and 3.3 with s = 2N): one block per position
// u reads its rows j (e_j = u) whole, coalesced, and writes the column-scaled
// sums to the work array in panel layout, complex column c = real columns
// (2c, 2c+1) at scratch[(c/W·L + u)·W + c%W] (W = 2^logW, the product's panel
// width).  Positions with no row get zeros.  The first FFT pass then reads
// the work array like the others.
__global__ void k_dense_scatter(const void* A, int64_t lda, int t, int a_f64, int split, const int* row_ptr,
                                const int* jlist, const float* cscale, int64_t L, int T, int logW,
                                cx<float>* scratch, int64_t s, int* err) {
  const int64_t u = blockIdx.x;
  const int beg = row_ptr[u], end = row_ptr[u + 1];
  for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < T; c += gridDim.y * blockDim.x) {
    float re = 0.f, im = 0.f;
    for (int q = beg; q < end; ++q) {
      const int64_t j = chk((int64_t)jlist[q], s, err);
      if (split) {
        const double x = reinterpret_cast<const double*>(A)[j * lda + c];
        const float hi = (float)x;
        re += hi;
        im += (float)(x - (double)hi);
      } else if (a_f64) {
        const double* row = reinterpret_cast<const double*>(A) + j * lda;
        if (2 * c < t) re += (float)row[2 * c];
        if (2 * c + 1 < t) im += (float)row[2 * c + 1];
      } else {
        const float* row = reinterpret_cast<const float*>(A) + j * lda;
        if (2 * c < t) re += row[2 * c];
        if (2 * c + 1 < t) im += row[2 * c + 1];
      }
    }
    cx<float> v;
    if (split) {
      v = mk<float>(re * cscale[c], im * cscale[c]);
    } else {
      v = mk<float>(2 * c < t ? re * cscale[2 * c] : 0.f, 2 * c + 1 < t ? im * cscale[2 * c + 1] : 0.f);
    }
    scratch[(((int64_t)(c >> logW) * L + u) << logW) + (c & ((1 << logW) - 1))] = v;
  }
}

int launch_dense_scatter(const PassArgs& a, cudaStream_t st) {
  const int nt = 256;
  int gy = (a.T + nt - 1) / nt;
  if (gy > 65535) gy = 65535;
  dim3 grid((unsigned)a.L, gy);
  k_dense_scatter<<<grid, nt, 0, st>>>(a.A, a.lda, a.t, a.a_f64, a.split, a.row_ptr, a.jlist, a.cscale, a.L,
                                       a.T, a.logW, reinterpret_cast<cx<float>*>(a.scratch), a.s_a, a.err);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // namespace qmc
