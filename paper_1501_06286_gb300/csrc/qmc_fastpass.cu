// qmc_fastpass.cu — register-resident pass kernels for the square pass
// lengths LP = P^2 (P = 16: 256 points, P = 32: 1024 points).
//
// Same passes as the generic kernel (see qmc_pass_kernel.cuh), with the
// LP-point transform done as P-point DFTs in registers:
//   point i = q + P·p.  Thread q holds x[q + P·p] for all p, does a P-point
//   DFT over p, multiplies by w_LP^{q·k_p}, and writes the P values to the
//   shared tile transposed; after one barrier thread k_p reads its P values
//   and does the second P-point DFT, ending with X[k_p + P·k_q] for all
//   k_q — which is again a stride-P set of points.  So the spectral pass
//   runs forward transform, spectrum product and inverse transform back to
//   back with one shared-memory exchange per transform, and every global
//   access is a stride-P sweep that the warp's lanes read as contiguous
//   rows of 8 complex columns.
#include "qmc_io.cuh"

namespace qmc {

namespace {

// 32-point DFT: n = q + 4m; DFT8 over m, twiddle by w32^{DIR q k1},
// DFT4 over q; X[k1 + 8 k2].  cos/sin(pi e/16) for e = 0..21.
template <int DIR>
__device__ __forceinline__ void dft32(cx<float>* v) {
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
__device__ __forceinline__ void dftP(cx<float>* v) {
  if constexpr (P == 16) dft16<DIR>(v);
  else dft32<DIR>(v);
}

constexpr int kFastM = 8;  // lines per block: 8 complex columns of one line group, or fewer columns

// Shared-tile index of (point i, line m): one padding row after every P
// points so that the transposed reads of neighbouring threads fall in
// different bank halves.
template <int P>
__device__ __forceinline__ int sidx(int i, int m) {
  return (i + i / P) * kFastM + m;
}

// LP = P^2 transform of the registers v (input x[t + P·p] at v[p], output
// X[t + P·k] at v[k]) for line m; all threads of the block participate.
template <int P, int DIR>
__device__ __forceinline__ void tile_fft(cx<float>* v, cx<float>* S, const cx<float>* tw, int t, int m) {
  dftP<P, DIR>(v);
#pragma unroll
  for (int k = 1; k < P; ++k) v[k] = twmul<DIR>(v[k], tw[t * k]);
#pragma unroll
  for (int k = 0; k < P; ++k) S[sidx<P>(k * P + t, m)] = v[k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < P; ++q) v[q] = S[sidx<P>(t * P + q, m)];
  dftP<P, DIR>(v);
  __syncthreads();
}

}  // namespace

enum FastMode : int { FM_FWD = 0, FM_SPECTRAL = 1, FM_INV = 2 };

template <int P, int LOAD, int STORE, int MODE>
__global__ void __launch_bounds__(P * kFastM, (P == 16 ? 6 : 2))
    k_fast(const __grid_constant__ PassArgs a) {
  constexpr int LP = P * P;
  constexpr int M = kFastM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* S = tw + LP;
  const int tid = threadIdx.x;
  const int logW = a.logW;
  const int W = 1 << logW;
  const int V = M >> logW;
  // thread -> (point sweep t, line m = v*W + w)
  int t, v, w;
  w = tid & (W - 1);
  if (MODE == FM_SPECTRAL) {      // points contiguous: w, then t, then line group
    t = (tid >> logW) & (P - 1);
    v = tid >> (logW + (P == 16 ? 4 : 5));
  } else {                        // points strided: w, then line group, then t
    v = (tid >> logW) & (V - 1);
    t = tid >> 3;
  }
  const int m = v * W + w;
  const int p = blockIdx.y;
  const int ag = blockIdx.x * V + v;
  const bool line_ok = ag < a.n_linegroups;
  const int c = (p << logW) + w;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += P * M) tw[k] = twL[(int64_t)k * tstep];
  }
  const int64_t rbase = (int64_t)ag * a.line_stride;
  const int64_t pstride = a.point_stride;
  cx<float> x[P];
  // ---- load the stride-P sweep of points t + P*k ------------------------
  if constexpr (LOAD == LD_GATHER_A) {
    gather_tile<float>(a, S, (LP + P) * M, blockIdx.x * V, V, logW, p,
                       [=](int i, int vv, int ww) { return sidx<P>(i, vv * W + ww); });
#pragma unroll
    for (int k = 0; k < P; ++k) x[k] = S[sidx<P>(t + P * k, m)];
    __syncthreads();  // S is rewritten by the transform
  } else {
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int i = t + P * k;
    const int64_t r = rbase + i * pstride;
    cx<float> val = mk<float>(0.f, 0.f);
    if (line_ok) {
      if constexpr (LOAD == LD_SCRATCH)
        val = reinterpret_cast<const cx<float>*>(a.scratch)[((int64_t)p * a.L + r) * W + w];
      else
        val = load_input<float, LOAD>(a, r, c);
    }
    x[k] = val;
  }
  __syncthreads();  // twiddle table ready
  }

  if (MODE == FM_FWD || MODE == FM_SPECTRAL) tile_fft<P, -1>(x, S, tw, t, m);
  if (MODE == FM_SPECTRAL) {
    const cx<float>* H = reinterpret_cast<const cx<float>*>(a.H);
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const cx<float> h = line_ok ? H[rbase + (t + P * k) * pstride] : mk<float>(0.f, 0.f);
      x[k] = a.mul == 1 ? x[k] * h : x[k] * conj(h);
    }
  }
  if (MODE == FM_INV || MODE == FM_SPECTRAL) tile_fft<P, +1>(x, S, tw, t, m);

  // ---- store the stride-P sweep -----------------------------------------
  float esum = 0.f;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int i = t + P * k;
    const int64_t r = rbase + i * pstride;
    cx<float> val = x[k];
    if (line_ok && a.twiddle) {
      const cx<float> wv = twL[(int64_t)ag * i];
      val = a.twiddle > 0 ? twmul<+1>(val, wv) : twmul<-1>(val, wv);
    }
    if constexpr (STORE == ST_SCRATCH) {
      if (line_ok) reinterpret_cast<cx<float>*>(a.scratch)[((int64_t)p * a.L + r) * W + w] = val;
    } else if constexpr (STORE == ST_OUT) {
      float contrib = 0.f;
      int64_t row = -1;
      if (line_ok && c < a.T) contrib = store_out<float>(a, r, c, val, esum, &row);
      if (a.row_mean) row_mean_add(a, contrib, row, w, W);
    } else if constexpr (STORE == ST_DA) {
      if (line_ok && c < a.T) store_da<float>(a, r, c, val);
    }
  }
  if constexpr (STORE == ST_OUT) {
    if (a.exp_sum) exp_sum_flush(a, esum);
  }
}

template <int P, int LOAD, int STORE, int MODE>
static int run_fast(const PassArgs& a, cudaStream_t st) {
  constexpr int LP = P * P;
  const size_t smem = sizeof(cx<float>) * ((size_t)LP + (size_t)(LP + P) * kFastM);
  static KernelSetup setup;
  if (const int rc = setup_kernel(k_fast<P, LOAD, STORE, MODE>, setup, smem, P * kFastM, nullptr)) return rc;
  const int V = kFastM >> a.logW;
  dim3 grid((a.n_linegroups + V - 1) / V, (a.T + (1 << a.logW) - 1) >> a.logW);
  k_fast<P, LOAD, STORE, MODE><<<grid, P * kFastM, smem, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int P>
static int dispatch_fast(const PassArgs& a, int load, int store, int mode, cudaStream_t st) {
  if (mode == FM_FWD && load == LD_GATHER_A && store == ST_SCRATCH)
    return run_fast<P, LD_GATHER_A, ST_SCRATCH, FM_FWD>(a, st);
  if (mode == FM_FWD && load == LD_PERM_G && store == ST_SCRATCH)
    return run_fast<P, LD_PERM_G, ST_SCRATCH, FM_FWD>(a, st);
  if (mode == FM_SPECTRAL && load == LD_SCRATCH && store == ST_SCRATCH)
    return run_fast<P, LD_SCRATCH, ST_SCRATCH, FM_SPECTRAL>(a, st);
  if (mode == FM_SPECTRAL && load == LD_GATHER_A && store == ST_OUT)
    return run_fast<P, LD_GATHER_A, ST_OUT, FM_SPECTRAL>(a, st);
  if (mode == FM_SPECTRAL && load == LD_PERM_G && store == ST_DA)
    return run_fast<P, LD_PERM_G, ST_DA, FM_SPECTRAL>(a, st);
  if (mode == FM_INV && load == LD_SCRATCH && store == ST_OUT)
    return run_fast<P, LD_SCRATCH, ST_OUT, FM_INV>(a, st);
  if (mode == FM_INV && load == LD_SCRATCH && store == ST_DA)
    return run_fast<P, LD_SCRATCH, ST_DA, FM_INV>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

bool fast_pass_supported(int LP) { return LP == 256 || LP == 1024; }

// Runs pass `a` with the register-resident kernel.  The pass is given by
// its flags: forward only (pass A), forward + spectrum + inverse (pass B,
// or a single pass), inverse only (pass C).  The tile is 8 lines: one
// panel of W <= 8 complex columns times 8/W line groups.
int launch_fast_pass(PassArgs a, int load, int store, cudaStream_t st) {
  int mode;
  if (a.fwd && a.inv) mode = FM_SPECTRAL;
  else if (a.fwd) mode = FM_FWD;
  else mode = FM_INV;
  if (a.logW > 3) return QMC_ERR_UNSUPPORTED;
  a.logV = 3 - a.logW;
  a.logM = 3;
  if (a.LP == 256) return dispatch_fast<16>(a, load, store, mode, st);
  if (a.LP == 1024) return dispatch_fast<32>(a, load, store, mode, st);
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
