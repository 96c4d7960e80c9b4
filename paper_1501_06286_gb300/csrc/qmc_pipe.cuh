// qmc_pipe.cuh — the persistent register-resident pass kernel for pass
// lengths LP = P^2 (P = 16 or 32): its transforms, shared-memory layout and
// tile loop, shared by the stand-alone launches (qmc_pipepass.cu) and the
// batch's persistent queue (qmc_batch.cu).
#pragma once
#include "qmc_async.cuh"
#include "qmc_io.cuh"

namespace qmc {

namespace {

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
      const cx<float> z = y[q][k1];
      if (e == 8) {                   // w32^8 = i
        y[q][k1] = muli<DIR>(z);
      } else if (e == 4 || e == 12) {  // c4·(±1 ± i)
        const float sr = e == 4 ? 1.f : -1.f;
        const float u = z.re * sr - DIR * z.im, v = z.im * sr + DIR * z.re;
        y[q][k1] = mk<float>(C[4] * u, C[4] * v);
      } else {
        const float wr = C[e], wi = DIR * S[e];
        y[q][k1] = mk<float>(z.re * wr - z.im * wi, z.re * wi + z.im * wr);
      }
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

// Twiddles w_LP^{t·k} of the middle stage, k = 1..P-1: from the block's
// table, or (TR = true) from registers the thread loaded once (t is fixed
// per thread for the whole kernel).
template <bool TR, int P>
struct MidTwiddles {
  const cx<float>* tw;
  int t;
  cx<float> r[TR ? P : 1];
  __device__ __forceinline__ void load() {
    if constexpr (TR) {
#pragma unroll
      for (int k = 1; k < P; ++k) r[k] = tw[t * k];
    }
  }
  __device__ __forceinline__ cx<float> operator()(int k) const {
    if constexpr (TR) return r[k];
    else return tw[t * k];
  }
};

template <int P, int DIR, typename TW>
__device__ __forceinline__ void pipe_fft(cx<float>* v, cx<float>* S, const TW& tw, int t, int w) {
  dftPp<P, DIR>(v);
#pragma unroll
  for (int k = 1; k < P; ++k) v[k] = twmul<DIR>(v[k], tw(k));
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

// Tiles of a work-array pass: line groups x 8-column panels.
inline int ntiles_of(const PassArgs& a) { return a.n_linegroups * ((a.T + 7) >> 3); }

// Tiles are numbered line group fastest: tile = p * n_linegroups + ag.
// A buffer slot holds the tile (padded layout) and two auxiliary arrays of
// LP entries fetched with it: the spectral pass's spectrum H and inter-pass
// twiddles w_L^{ag·i}, or the un-permute pass's output rows.
template <int P, int MODE, int STORE>
struct PipeSlot {
  static constexpr int LP = P * P;
  static constexpr int SZ = (LP + P) * 8;   // padded tile (complex elements)
  // spectral: H and twiddles (2 LP complex); the other passes: none
  static constexpr int AUX = MODE == 1 ? 2 * LP : 0;
  static constexpr int SLOT = SZ + AUX;
};

// SPEC selects a specialised variant:
//   spectral pass: SPEC = 1 multiplies by H, 2 by conj(H); its points are
//     contiguous rows and its store twiddle is w_L^{+ag·i};
//   un-permute pass (ST_OUT): SPEC = 1 is the plain FP32 store (no split
//     columns, no epilogues), 0 the general one;
//   adjoint last pass (ST_DA): SPEC = 0.
// Middle-stage twiddles of the P = 16 work-array passes held in registers
// (1) or read from the block's table (0).
#ifndef QMC_TW_REGS
#define QMC_TW_REGS 1
#endif

// P = 32 tiles (64 KB) with one shared buffer and two resident blocks per
// SM (1), or double-buffered with one block (0).
#ifndef QMC_PIPE32_SINGLE
#define QMC_PIPE32_SINGLE 1
#endif
template <int P>
__host__ __device__ constexpr int pipe_buffers() { return (P == 32 && QMC_PIPE32_SINGLE) ? 1 : 2; }

// Resident blocks per SM the P = 16 kernels are compiled for (register cap).
#ifndef QMC_PIPE_LEAN_OUT_BLOCKS
#define QMC_PIPE_LEAN_OUT_BLOCKS 5
#endif
template <int P, int MODE, int STORE, int SPEC>
constexpr int pipe_min_blocks() {
  if (P != 16) return QMC_PIPE32_SINGLE ? 2 : 1;
  if (MODE == 1) return QMC_TW_REGS ? 4 : 5;
  if (STORE == ST_OUT && SPEC == 1) return QMC_TW_REGS ? 4 : QMC_PIPE_LEAN_OUT_BLOCKS;
  return QMC_TW_REGS ? 5 : 6;
}

// Packed rows: ap[(p·s + q)·8 + w] = complex column 8p + w of row
// j = sp_row[q], scaled like the scatter-add's (real columns 2c, 2c+1; or
// the hi/lo halves of FP64 column c in split precision); zero past the
// last column; entry q, complex columns c0, c0 + cstep, ...
__device__ __forceinline__ void sparse_pack_row(const PassArgs& a, int q, int ncols, int c0, int cstep) {
  const int64_t j = chk((int64_t)a.sp_row[q], a.s_a, a.err);
  cx<float>* ap = reinterpret_cast<cx<float>*>(a.sp_ap);
  for (int c = c0; c < ncols; c += cstep) {
    cx<float> v = mk<float>(0.f, 0.f);
    if (c < a.T) {
      if (a.split) {
        const double x = reinterpret_cast<const double*>(a.A)[j * a.lda + c];
        const float hi = (float)x;
        v = mk<float>(hi * a.cscale[c], (float)(x - (double)hi) * a.cscale[c]);
      } else if (a.a_f64) {
        const double* row = reinterpret_cast<const double*>(a.A) + j * a.lda;
        v.re = (float)row[2 * c] * a.cscale[2 * c];
        if (2 * c + 1 < a.t) v.im = (float)row[2 * c + 1] * a.cscale[2 * c + 1];
      } else {
        const float* row = reinterpret_cast<const float*>(a.A) + j * a.lda;
        v.re = row[2 * c] * a.cscale[2 * c];
        if (2 * c + 1 < a.t) v.im = row[2 * c + 1] * a.cscale[2 * c + 1];
      }
    }
    ap[((int64_t)(c >> 3) * a.sp_s + q) * 8 + (c & 7)] = v;
  }
}

// The persistent pass kernel; its tile loop (qmc_pipe_body.inc) is shared
// with the batch's persistent queue, which runs it on chunks of tiles.
template <int P, int MODE, int STORE, int SPEC>
__global__ void __launch_bounds__(P * 8, (pipe_min_blocks<P, MODE, STORE, SPEC>()))
    k_pipe(const __grid_constant__ PassArgs a, int ntiles) {
  auto first_of = [&]() -> int { return (int)blockIdx.x; };
  auto step_of = [&]() -> int { return (int)gridDim.x; };
#include "qmc_pipe_body.inc"
}

}  // namespace qmc
