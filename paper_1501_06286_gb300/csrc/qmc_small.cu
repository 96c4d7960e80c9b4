// qmc_small.cu — the whole forward product of a small plan in one launch:
// single-pass lengths (L <= 1024) and at most one panel of columns
// (t <= 16).  The block first forms its columns' sums and l1 norms (row 0
// = φ(0)·Σ_j A_j, Section 2.1, and the power-of-two column scales), then
// runs the single pass: scatter-add, FFT, ×H, inverse FFT, un-permute.
// Products this small are bound by launch latency, and this replaces the
// three launches of the general path (two for the column statistics) by one.
#include <math.h>

#include "qmc_pass_kernel.cuh"

namespace qmc {

namespace {

constexpr int kSmallMaxT = 16;

__global__ void __launch_bounds__(512) k_small(const __grid_constant__ PassArgs a, double phi0, int has_row0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float scale_s[kSmallMaxT], inv_s[kSmallMaxT];
  __shared__ double red_sum[16][kSmallMaxT], red_l1[16][kSmallMaxT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // FP64 column sums and l1 norms over the s rows of A: every thread takes
  // rows j = tid, tid + nt, ... of all t columns (t <= 16), then a fixed-order
  // reduction over lanes and warps
  for (int k0 = 0; k0 < a.t; k0 += 4) {  // four columns at a time
    double sum[4] = {0.0, 0.0, 0.0, 0.0}, l1[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < a.s_a; j += blockDim.x) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q;
        if (k < a.t) {
          const double v = a.a_f64 ? reinterpret_cast<const double*>(a.A)[(int64_t)j * a.lda + k]
                                   : (double)reinterpret_cast<const float*>(a.A)[(int64_t)j * a.lda + k];
          sum[q] += v;
          l1[q] += fabs(v);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      for (int off = 16; off > 0; off >>= 1) {
        sum[q] += __shfl_xor_sync(0xffffffffu, sum[q], off);
        l1[q] += __shfl_xor_sync(0xffffffffu, l1[q], off);
      }
      if (lane == 0 && k0 + q < a.t) { red_sum[warp][k0 + q] = sum[q]; red_l1[warp][k0 + q] = l1[q]; }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < a.t; k += blockDim.x) {
    double sum = 0.0, l1 = 0.0;
    for (int w8 = 0; w8 < nwarps; ++w8) { sum += red_sum[w8][k]; l1 += red_l1[w8][k]; }
    {
      if (l1 > 0.0 && isfinite(l1)) {
        const int e = max(-100, min(100, ilogb(l1)));
        scale_s[k] = (float)ldexp(1.0, -e);
        inv_s[k] = (float)ldexp(1.0, e);
      } else {
        scale_s[k] = 0.f;
        inv_s[k] = 0.f;
      }
      if (has_row0) {
        float b0 = (float)(phi0 * sum);
        if (a.col_off || a.out_exp) b0 = affine_out(a, k, b0);
        a.out[k] = b0;  // row 0 is output row 0
        if (a.exp_sum) atomicAdd(a.exp_sum, exp((double)b0));
      }
    }
  }
  __syncthreads();
  PassArgs b = a;
  b.cscale = scale_s;
  b.cinv = inv_s;
  pass_tile<float, LD_GATHER_A, ST_OUT>(b, 0, 0, smem_raw);
}

}  // namespace

// Forward product of a single-pass plan with t <= 16 in one launch;
// QMC_ERR_UNSUPPORTED when the plan or call needs the general path.
int launch_small_product(const Plan& p, const PassSpec& sp, cudaStream_t st) {
  const PassArgs& a = sp.a;
  if (p.L2 != 1 || a.t > kSmallMaxT || a.T > 8 || a.split || a.row_mean || sp.load != LD_GATHER_A ||
      sp.store != ST_OUT || a.logV != 0)
    return QMC_ERR_UNSUPPORTED;
  const int items = a.LP << a.logM;
  int nt = (items + kEPT - 1) / kEPT;
  nt = ((nt + 31) / 32) * 32;
  if (nt > 512) return QMC_ERR_UNSUPPORTED;
  // latency-bound: more threads than the throughput kernels use, so that
  // each FFT stage is a few elements per thread
  nt = max(nt, min(256, ((items / 2 + 31) / 32) * 32));
  if (nt < 32) nt = 32;
  const bool rader = a.nst == 1 && (int)(a.rbits & 31u) == kRader257;
  const size_t smem = sizeof(cx<float>) * ((size_t)a.LP + 2 * (size_t)items +
                                           (rader ? 256 + 2 * ((size_t)1 << a.logM) : 0));
  static KernelSetup setup;
  if (const int rc = setup_kernel(k_small, setup, smem, nt, nullptr)) return rc;
  PassArgs b = a;
  b.s_a = p.s;
  k_small<<<1, nt, smem, st>>>(b, p.phi0, p.has_row0);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // namespace qmc
