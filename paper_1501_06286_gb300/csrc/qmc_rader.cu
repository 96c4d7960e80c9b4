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
// t + 16k of a column, one shared-memory transpose per transform, its
// middle twiddles in registers.
#include "qmc_async.cuh"
#include "qmc_io.cuh"

namespace qmc {

namespace {

constexpr int kRP = 16;          // 256 = 16 x 16
constexpr int kRLines = 8;       // columns per tile
constexpr int kRNT = kRP * kRLines;
constexpr int kXS = 257 * kRLines;            // the line, natural order
constexpr int kSZ = (256 + kRP) * kRLines;    // padded transpose area (>= kXS)
constexpr int kSlot = kSZ + 2 * 257 + 2;      // tile/scratch + H + twiddles (16-byte multiple)

__device__ __forceinline__ int ridx(int i, int w) { return (i + i / kRP) * kRLines + w; }

// FFT_256 of one column; thread t holds points t + 16k on entry and exit;
// twr[k] = w_256^{t·k} in registers; S is the padded transpose area.
template <int DIR>
__device__ __forceinline__ void fft256(cx<float>* v, cx<float>* S, const cx<float>* twr, int t, int w) {
  dft16<DIR>(v);
#pragma unroll
  for (int k = 1; k < kRP; ++k) v[k] = twmul<DIR>(v[k], twr[k]);
#pragma unroll
  for (int k = 0; k < kRP; ++k) S[ridx(k * kRP + t, w)] = v[k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kRP; ++q) v[q] = S[ridx(t * kRP + q, w)];
  dft16<DIR>(v);
  __syncthreads();
}

// DFT_257 (direction DIR) of the 8 columns held in xs[n*8 + w]; output
// point n of column w goes to store(n, value).  The transposes reuse xs's
// storage once every thread has read its inputs.
template <int DIR, typename Store>
__device__ __forceinline__ void dft257(cx<float>* xs, const cx<float>* twr, const cx<float>* what,
                                       const int16_t* pin, const int16_t* pout, int t, int w, Store store) {
  const cx<float> x0 = xs[w];
  cx<float> v[kRP];
#pragma unroll
  for (int k = 0; k < kRP; ++k) v[k] = xs[(int)pin[t + kRP * k] * kRLines + w];
  __syncthreads();                 // xs is free: its storage becomes the transpose area
  fft256<-1>(v, xs, twr, t, w);    // U at points t + 16k
  const cx<float> u0 = v[0];       // U[0] = Σ_a u_a, held by thread t = 0
#pragma unroll
  for (int k = 0; k < kRP; ++k) v[k] = v[k] * what[t + kRP * k];
  fft256<+1>(v, xs, twr, t, w);    // (u ⊛ w)_b at b = t + 16k; ends with a barrier
#pragma unroll
  for (int k = 0; k < kRP; ++k) store((int)pout[t + kRP * k], x0 + v[k]);
  if (t == 0) store(0, x0 + u0);
  __syncthreads();
}

// Persistent: tile = one line (k1) of one 8-column panel, line fastest; the
// next tile's 257 rows (one contiguous 16 KB run), spectrum entries and
// store twiddles are copied with cp.async while this one is transformed.
template <int MUL>
__global__ void __launch_bounds__(kRNT, 4) k_rader_spectral(const __grid_constant__ PassArgs a, int ntiles) {
  __shared__ __align__(16) cx<float> what_f[256], what_i[256];
  __shared__ int16_t pin[256], pout[256];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* slots = reinterpret_cast<cx<float>*>(smem_raw);
  const int tid = threadIdx.x;
  const int w = tid & 7, t = tid >> 3;
  const cx<float>* tab = reinterpret_cast<const cx<float>*>(a.rader);
  for (int k = tid; k < 256; k += kRNT) {
    what_f[k] = tab[256 + k];
    what_i[k] = tab[512 + k];
    pin[k] = a.rader_perm[k];
    pout[k] = a.rader_perm[256 + k];
  }
  cx<float> twr[kRP];  // w_256^{t·k}, fixed per thread
#pragma unroll
  for (int k = 0; k < kRP; ++k) twr[k] = tab[t * k];
  const cx<float>* scratch = reinterpret_cast<const cx<float>*>(a.scratch);
  const cx<float>* H = reinterpret_cast<const cx<float>*>(a.H);
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  const int nlg = a.n_linegroups;

  auto prefetch = [&](int tile, cx<float>* dst) {
    const int ag = tile % nlg, p = tile / nlg;
    const int64_t rbase = (int64_t)ag * a.line_stride;
    const cx<float>* src = scratch + ((int64_t)p * a.L + rbase) * kRLines;
    for (int c = tid; c < kXS / 2; c += kRNT) cp_async16(dst + 2 * c, src + 2 * c);
    cx<float>* hs = dst + kSZ;
    cx<float>* ts = hs + 257;
    for (int i = tid; i < 257; i += kRNT) {
      cp_async8(hs + i, H + rbase + i);
      cp_async8(ts + i, twL + (int64_t)ag * i);
    }
    cp_async_commit();
  };

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, slots);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    cx<float>* xs = slots + (it & 1) * kSlot;
    const cx<float>* hs = xs + kSZ;
    const cx<float>* ts = hs + 257;
    const int next = tile + gridDim.x;
    if (next < ntiles) prefetch(next, slots + ((it + 1) & 1) * kSlot);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();  // this tile has landed (and, first time round, the tables)
    // forward DFT, its outputs multiplied by H (or conj(H)) as they land
    dft257<-1>(xs, twr, what_f, pin, pout, t, w, [&](int n, cx<float> x) {
      const cx<float> h = hs[n];
      xs[n * kRLines + w] = MUL == 1 ? x * h : x * conj(h);
    });
    // inverse DFT, its outputs twiddled and stored to the work array (the
    // 64-byte rows of the line's points, in Rader's output order); its
    // closing barrier frees the slot, the prefetch target two tiles on
    const int ag = tile % nlg, p = tile / nlg;
    cx<float>* dst = reinterpret_cast<cx<float>*>(a.scratch) + ((int64_t)p * a.L + (int64_t)ag * a.line_stride) * kRLines;
    dft257<+1>(xs, twr, what_i, pin, pout, t, w, [&](int n, cx<float> x) {
      dst[n * kRLines + w] = twmul<+1>(x, ts[n]);
    });
  }
  cp_async_wait<0>();
}

template <int MUL>
int run_rader(const PassArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(cx<float>) * 2 * (size_t)kSlot;
  static KernelSetup setup;
  int grid = 0;
  if (const int rc = setup_kernel(k_rader_spectral<MUL>, setup, smem, kRNT, &grid)) return rc;
  const int ntiles = a.n_linegroups * ((a.T + 7) >> 3);
  if (grid > ntiles) grid = ntiles;
  k_rader_spectral<MUL><<<grid, kRNT, smem, st>>>(a, ntiles);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // namespace

// Spectral pass of length 257 over 8-column panels (contiguous points,
// store twiddle w_L^{+ag·i}).
int launch_rader_spectral(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (a.LP != 257 || !(a.fwd && a.inv) || a.logW != 3 || load != LD_SCRATCH || store != ST_SCRATCH ||
      a.point_stride != 1 || a.twiddle != 1 || !a.rader || !a.rader_perm)
    return QMC_ERR_UNSUPPORTED;
  if (a.mul == 1) return run_rader<1>(a, st);
  if (a.mul == 2) return run_rader<2>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
