// qmc_fast.cuh — the transforms of the register-resident tile of the square
// pass lengths LP = P^2 (P = 16: 256 points, P = 32: 1024 points), whose
// tile (qmc_fast_body.inc) the stand-alone kernel k_fast (qmc_fastpass.cu)
// and the batch's persistent queue run.
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
#pragma once
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

// Shared-tile index of (point i, line m) for a tile of M lines: one padding
// row after every P points so that the transposed reads of neighbouring
// threads fall in different bank halves.
template <int P, int M = kFastM>
__device__ __forceinline__ int sidx(int i, int m) {
  return (i + i / P) * M + m;
}

// LP = P^2 transform of the registers v (input x[t + P·p] at v[p], output
// X[t + P·k] at v[k]) for line m; all threads of the block participate.
template <int P, int DIR, int M = kFastM>
__device__ __forceinline__ void tile_fft(cx<float>* v, cx<float>* S, const cx<float>* tw, int t, int m) {
  dftP<P, DIR>(v);
#pragma unroll
  for (int k = 1; k < P; ++k) v[k] = twmul<DIR>(v[k], tw[t * k]);
#pragma unroll
  for (int k = 0; k < P; ++k) S[sidx<P, M>(k * P + t, m)] = v[k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < P; ++q) v[q] = S[sidx<P, M>(t * P + q, m)];
  dftP<P, DIR>(v);
  __syncthreads();
}

}  // namespace

enum FastMode : int { FM_FWD = 0, FM_SPECTRAL = 1, FM_INV = 2 };

}  // namespace qmc
