// qmc_rader.cu — register-resident spectral pass for pass length 257 (the
// prime factor of L = 2^16 - 1 = 255·257 of polynomial lattices with
// m = 16): forward DFT_257, spectrum product, inverse DFT_257, inter-pass
// twiddle, for one line (k1) of 8 complex columns per block.
//
// Each DFT_257 is Rader's algorithm with primitive root 3: u_a = x[3^a],
// X[0] = x_0 + Σ_a u_a and X[3^{-b}] = x_0 + (u ⊛ w)_b, the 256-point
// cyclic convolution done as a forward FFT_256, a product with the
// precomputed DFT of w (scaled by 1/256), and an inverse FFT_256.  The
// FFT_256 is the 16 x 16 register transform: thread t holds points
// t + 16k of a column, one shared-memory transpose per transform.
#include "qmc_io.cuh"

namespace qmc {

namespace {

constexpr int kRP = 16;          // 256 = 16 x 16
constexpr int kRLines = 8;       // columns per block

__device__ __forceinline__ int ridx(int i, int w) { return (i + i / kRP) * kRLines + w; }

template <int DIR>
__device__ __forceinline__ void fft256(cx<float>* v, cx<float>* S, const cx<float>* tw, int t, int w) {
  dft16<DIR>(v);
#pragma unroll
  for (int k = 1; k < kRP; ++k) v[k] = twmul<DIR>(v[k], tw[t * k]);
#pragma unroll
  for (int k = 0; k < kRP; ++k) S[ridx(k * kRP + t, w)] = v[k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kRP; ++q) v[q] = S[ridx(t * kRP + q, w)];
  dft16<DIR>(v);
  __syncthreads();
}

// In-place DFT_257 (direction DIR) of the 8 columns held in xs[n*8 + w].
template <int DIR>
__device__ __forceinline__ void dft257(cx<float>* xs, cx<float>* S, const cx<float>* tw256,
                                       const cx<float>* what, const int16_t* pin, const int16_t* pout,
                                       int t, int w) {
  const cx<float> x0 = xs[w];
  cx<float> v[kRP];
#pragma unroll
  for (int k = 0; k < kRP; ++k) v[k] = xs[(int)pin[t + kRP * k] * kRLines + w];
  fft256<-1>(v, S, tw256, t, w);  // U at points t + 16k (contains the barrier before xs is rewritten)
  const cx<float> u0 = v[0];      // U[0] = Σ_a u_a, held by thread t = 0
#pragma unroll
  for (int k = 0; k < kRP; ++k) v[k] = v[k] * what[t + kRP * k];
  fft256<+1>(v, S, tw256, t, w);  // (u ⊛ w)_b at b = t + 16k
#pragma unroll
  for (int k = 0; k < kRP; ++k) xs[(int)pout[t + kRP * k] * kRLines + w] = x0 + v[k];
  if (t == 0) xs[w] = x0 + u0;
  __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(kRP * kRLines, 5) k_rader_spectral(const __grid_constant__ PassArgs a) {
  __shared__ cx<float> tw256[256], what_f[256], what_i[256];
  __shared__ int16_t pin[256], pout[256];
  __shared__ cx<float> xs[257 * kRLines];
  __shared__ cx<float> S[(256 + kRP) * kRLines];
  const int tid = threadIdx.x;
  const int w = tid & 7, t = tid >> 3;
  const int ag = blockIdx.x, p = blockIdx.y;
  const cx<float>* tab = reinterpret_cast<const cx<float>*>(a.rader);
  for (int k = tid; k < 256; k += blockDim.x) {
    tw256[k] = tab[k];
    what_f[k] = tab[256 + k];
    what_i[k] = tab[512 + k];
    pin[k] = a.rader_perm[k];
    pout[k] = a.rader_perm[256 + k];
  }
  const int64_t rbase = (int64_t)ag * a.line_stride;
  const cx<float>* src = reinterpret_cast<const cx<float>*>(a.scratch) + ((int64_t)p * a.L + rbase) * 8;
  for (int e = tid; e < 257 * kRLines; e += blockDim.x) xs[e] = ld_cg(src + e);  // rows contiguous
  __syncthreads();
  dft257<-1>(xs, S, tw256, what_f, pin, pout, t, w);
  const cx<float>* H = reinterpret_cast<const cx<float>*>(a.H) + rbase;
  for (int e = tid; e < 257 * kRLines; e += blockDim.x) {
    const cx<float> h = H[e >> 3];
    xs[e] = a.mul == 1 ? xs[e] * h : xs[e] * conj(h);
  }
  __syncthreads();
  dft257<+1>(xs, S, tw256, what_i, pin, pout, t, w);
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  cx<float>* dst = reinterpret_cast<cx<float>*>(a.scratch) + ((int64_t)p * a.L + rbase) * 8;
  for (int e = tid; e < 257 * kRLines; e += blockDim.x) {
    cx<float> val = xs[e];
    if (a.twiddle) {
      const cx<float> wv = twL[(int64_t)ag * (e >> 3)];
      val = a.twiddle > 0 ? twmul<+1>(val, wv) : twmul<-1>(val, wv);
    }
    dst[e] = val;
  }
}

// Spectral pass of length 257 over 8-column panels.
int launch_rader_spectral(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (a.LP != 257 || !(a.fwd && a.inv) || a.logW != 3 || load != LD_SCRATCH || store != ST_SCRATCH ||
      a.point_stride != 1 || !a.rader || !a.rader_perm)
    return QMC_ERR_UNSUPPORTED;
  dim3 grid(a.n_linegroups, (a.T + 7) >> 3);
  k_rader_spectral<<<grid, kRP * kRLines, 0, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // namespace qmc
