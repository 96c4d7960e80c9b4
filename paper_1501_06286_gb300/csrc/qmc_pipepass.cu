// qmc_pipepass.cu — persistent, double-buffered version of the
// register-resident pass kernel for the work-array passes (spectral pass B
// and inverse/un-permute pass C, forward and adjoint), pass lengths
// LP = P^2 with P = 16 or 32, panels of 8 complex columns.
//
// Each block loops over tiles (one line group of one panel: LP points x 8
// columns).  While it transforms tile i it has already issued the 16-byte
// cp.async copies of tile i+1 into the other shared buffer, so HBM reads
// stay in flight independently of how many blocks fit on an SM.  The
// shared buffer a tile lands in has the padded layout of the transposes and
// serves as their scratch, so a block needs two tile buffers and no more.
#include "qmc_io.cuh"

namespace qmc {

namespace {

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 32-point DFT (same decomposition as in qmc_fastpass.cu): n = q + 4m.
template <int DIR>
__device__ __forceinline__ void dft32p(cx<float>* v) {
  constexpr float C[22] = {1.f, 0.98078528040323044913f, 0.92387953251128675613f,
                           0.83146961230254523708f, 0.70710678118654752440f, 0.55557023301960222474f,
                           0.38268343236508977173f, 0.19509032201612826785f, 0.f,
                           -0.19509032201612826785f, -0.38268343236508977173f, -0.55557023301960222474f,
                           -0.70710678118654752440f, -0.83146961230254523708f, -0.92387953251128675613f,
                           -0.98078528040323044913f, -1.f, -0.98078528040323044913f,
                           -0.92387953251128675613f, -0.83146961230254523708f, -0.70710678118654752440f,
                           -0.55557023301960222474f};
  constexpr float S[22] = {0.f, 0.19509032201612826785f, 0.38268343236508977173f,
                           0.55557023301960222474f, 0.70710678118654752440f, 0.83146961230254523708f,
                           0.92387953251128675613f, 0.98078528040323044913f, 1.f,
                           0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                           0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                           0.19509032201612826785f, 0.f, -0.19509032201612826785f,
                           -0.38268343236508977173f, -0.55557023301960222474f,
                           -0.70710678118654752440f, -0.83146961230254523708f};
  cx<float> y[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int m = 0; m < 8; ++m) y[q][m] = v[q + 4 * m];
    dft8<DIR>(y[q]);
  }
#pragma unroll
  for (int q = 1; q < 4; ++q) {
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) {
      const int e = q * k1;
      const float wr = C[e], wi = DIR * S[e];
      const cx<float> z = y[q][k1];
      y[q][k1] = mk<float>(z.re * wr - z.im * wi, z.re * wi + z.im * wr);
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    cx<float> a0 = y[0][k1], a1 = y[1][k1], a2 = y[2][k1], a3 = y[3][k1];
    dft4<DIR>(a0, a1, a2, a3);
    v[k1] = a0; v[k1 + 8] = a1; v[k1 + 16] = a2; v[k1 + 24] = a3;
  }
}

template <int P, int DIR>
__device__ __forceinline__ void dftPp(cx<float>* v) {
  if constexpr (P == 16) dft16<DIR>(v);
  else dft32p<DIR>(v);
}

// padded tile index of (point i, column w), 8 columns per point row and one
// padding row after every P points
template <int P>
__device__ __forceinline__ int pidx(int i, int w) { return (i + i / P) * 8 + w; }

template <int P, int DIR>
__device__ __forceinline__ void pipe_fft(cx<float>* v, cx<float>* S, const cx<float>* tw, int t, int w) {
  dftPp<P, DIR>(v);
#pragma unroll
  for (int k = 1; k < P; ++k) v[k] = twmul<DIR>(v[k], tw[t * k]);
#pragma unroll
  for (int k = 0; k < P; ++k) S[pidx<P>(k * P + t, w)] = v[k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < P; ++q) v[q] = S[pidx<P>(t * P + q, w)];
  dftPp<P, DIR>(v);
  __syncthreads();
}

}  // namespace

enum PipeMode : int { PM_SPECTRAL = 1, PM_INV = 2 };

// Tiles are numbered line group fastest: tile = p * n_linegroups + ag.
template <int P, int MODE, int STORE>
__global__ void __launch_bounds__(P * 8, (P == 16 ? 6 : 1))
    k_pipe(const __grid_constant__ PassArgs a, int ntiles) {
  constexpr int LP = P * P;
  constexpr int SZ = (LP + P) * 8;
  constexpr int NT = P * 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* bufs = tw + LP;
  const int tid = threadIdx.x;
  const int w = tid & 7, t = tid >> 3;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += NT) tw[k] = twL[(int64_t)k * tstep];
  }
  const cx<float>* scratch_in = reinterpret_cast<const cx<float>*>(a.scratch);
  const int64_t pst = (int64_t)a.point_stride * 8;  // complex elements between points
  const int nlg = a.n_linegroups;

  auto prefetch = [&](int tile, cx<float>* dst) {
    const int ag = tile % nlg, p = tile / nlg;
    const cx<float>* base = scratch_in + ((int64_t)p * a.L + (int64_t)ag * a.line_stride) * 8;
#pragma unroll
    for (int q = 0; q < LP * 4 / NT; ++q) {
      const int c = tid + q * NT;        // 16-byte chunk: point c/4, columns 2*(c%4), +1
      const int i = c >> 2, part = (c & 3) * 2;
      cp_async16(dst + pidx<P>(i, part), base + i * pst + part);
    }
    cp_async_commit();
  };

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, bufs);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    cx<float>* cur = bufs + (it & 1) * SZ;
    cx<float>* nxt = bufs + ((it + 1) & 1) * SZ;
    const int next = tile + gridDim.x;
    if (next < ntiles) prefetch(next, nxt);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    cx<float> x[P];
#pragma unroll
    for (int k = 0; k < P; ++k) x[k] = cur[pidx<P>(t + P * k, w)];
    __syncthreads();

    const int ag = tile % nlg, p = tile / nlg;
    const int64_t rbase = (int64_t)ag * a.line_stride;
    if (MODE == PM_SPECTRAL) {
      pipe_fft<P, -1>(x, cur, tw, t, w);
      const cx<float>* H = reinterpret_cast<const cx<float>*>(a.H) + rbase;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const cx<float> h = H[(t + P * k) * a.point_stride];
        x[k] = a.mul == 1 ? x[k] * h : x[k] * conj(h);
      }
    }
    pipe_fft<P, +1>(x, cur, tw, t, w);

    const int c = (p << 3) + w;
    if constexpr (STORE == ST_SCRATCH) {
      cx<float>* obase = reinterpret_cast<cx<float>*>(a.scratch) + ((int64_t)p * a.L + rbase) * 8 + w;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int i = t + P * k;
        cx<float> val = x[k];
        if (a.twiddle) {
          const cx<float> wv = twL[(int64_t)ag * i];
          val = a.twiddle > 0 ? twmul<+1>(val, wv) : twmul<-1>(val, wv);
        }
        obase[i * pst] = val;
      }
    } else if constexpr (STORE == ST_OUT) {
      float esum = 0.f;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int64_t r = rbase + (int64_t)(t + P * k) * a.point_stride;
        float contrib = 0.f;
        int64_t row = -1;
        if (c < a.T) contrib = store_out<float>(a, r, c, x[k], esum, &row);
        if (a.row_mean) row_mean_add(a, contrib, row, w, 8);
      }
      if (a.exp_sum) exp_sum_flush(a, esum);
    } else if constexpr (STORE == ST_DA) {
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int64_t r = rbase + (int64_t)(t + P * k) * a.point_stride;
        if (c < a.T) store_da<float>(a, r, c, x[k]);
      }
    }
  }
  cp_async_wait<0>();
}

template <int P, int MODE, int STORE>
static int run_pipe(const PassArgs& a, cudaStream_t st) {
  constexpr int LP = P * P;
  const size_t smem = sizeof(cx<float>) * ((size_t)LP + 2 * (size_t)(LP + P) * 8);
  static size_t configured = 48 * 1024;
  static int blocks_per_sm = 0, sms = 0;
  if (smem > configured) {
    if (cudaFuncSetAttribute(k_pipe<P, MODE, STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return QMC_ERR_UNSUPPORTED;
    }
    configured = smem;
  }
  if (!blocks_per_sm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_pipe<P, MODE, STORE>, P * 8,
                                                      smem) != cudaSuccess ||
        blocks_per_sm < 1) {
      cudaGetLastError();
      blocks_per_sm = 0;
      return QMC_ERR_UNSUPPORTED;
    }
  }
  const int ntiles = a.n_linegroups * ((a.T + 7) >> 3);
  int grid = sms * blocks_per_sm;
  if (grid > ntiles) grid = ntiles;
  k_pipe<P, MODE, STORE><<<grid, P * 8, smem, st>>>(a, ntiles);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

// Passes that read the work array (spectral pass or inverse/un-permute
// pass) with panels of 8 columns; anything else is QMC_ERR_UNSUPPORTED and
// the caller uses another kernel.
int launch_pipe_pass(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (load != LD_SCRATCH || a.logW != 3) return QMC_ERR_UNSUPPORTED;
  const bool spectral = a.fwd && a.inv;
  const bool inv_only = !a.fwd && a.inv;
  if (a.LP == 256) {
    if (spectral && store == ST_SCRATCH) return run_pipe<16, PM_SPECTRAL, ST_SCRATCH>(a, st);
    if (inv_only && store == ST_OUT) return run_pipe<16, PM_INV, ST_OUT>(a, st);
    if (inv_only && store == ST_DA) return run_pipe<16, PM_INV, ST_DA>(a, st);
  } else if (a.LP == 1024) {
    if (spectral && store == ST_SCRATCH) return run_pipe<32, PM_SPECTRAL, ST_SCRATCH>(a, st);
    if (inv_only && store == ST_OUT) return run_pipe<32, PM_INV, ST_OUT>(a, st);
    if (inv_only && store == ST_DA) return run_pipe<32, PM_INV, ST_DA>(a, st);
  }
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
