// qmc_pqpipe.cuh — shapes, A staging helpers and the tile-loop kernels of
// the persistent P x Q passes that the batch's persistent queue runs too:
// the un-permute pass, the first pass from the padded gather table and
// the term-by-term first pass (the loops themselves are the textual
// bodies qmc_pqpipe_out_body.inc, qmc_pqpipe_gather_body.inc and
// qmc_pq_direct_body.inc).
#pragma once
#include "qmc_async.cuh"
#include "qmc_io.cuh"
#include "qmc_pq.cuh"

namespace qmc {

using namespace pq;

namespace {

template <int P, int Q>
struct PqPipeShape {
  static constexpr int LP = P * Q;
  static constexpr int TPL = P > Q ? P : Q;
  static constexpr int NT = ((TPL * kLines + 31) / 32) * 32;
  static constexpr int MINB = LP >= 512 ? 2 : 3;  // resident blocks the registers are sized for
  static constexpr int SZ = (LP + LP / Q) * kLines;  // padded tile (complex)
  // un-permute slot: tile + output rows (LP ints, rounded to 16 bytes)
  static constexpr int ROWS_CX = ((LP + 3) / 4) * 2;
  static constexpr int OUT_SLOT = SZ + ROWS_CX;
  // adjoint last pass: tile + the CSR bounds row_ptr[r], row_ptr[r + 1]
  static constexpr int DA_SLOT = SZ + 2 * ROWS_CX;
  // first-pass slot: staged A segments + twiddles + point indices, rounded
  // to 16 bytes so that the second slot's staging area stays aligned
  static constexpr int STG = kGatherMax * kLines;
  static constexpr int GATHER_SLOT = ((STG + LP + kGatherMax / 2 + 1) / 2) * 2;
};

// ---------------------------------------------------------------------------
// Last pass: inverse P x Q transform of each line, then
//   KIND 0, 1: out[out_row(r)][2c, 2c+1] = value / column scale (KIND 1 adds
//              Σ exp(B) over the block's outputs to *exp_sum once, at the end);
//   KIND 2:    the adjoint's dA[j] = value / column scale (+ φ(0)·G_0) for
//              every j with e_j = r, from the CSR bounds staged with the tile.
// ---------------------------------------------------------------------------
template <int P, int Q, int KIND>
__global__ void __launch_bounds__(PqPipeShape<P, Q>::NT, PqPipeShape<P, Q>::MINB) k_pqpipe_out(const __grid_constant__ PassArgs a,
                                                                     int ntiles) {
  auto first_of = [&]() -> int { return (int)blockIdx.x; };
  auto step_of = [&]() -> int { return (int)gridDim.x; };
#include "qmc_pqpipe_out_body.inc"
}

// ---------------------------------------------------------------------------
// Staging of A's rows in the first-pass kernels.  Entry e of a tile holds
// the 64-byte piece of its row that the tile's panel p needs, copied in
// four 16-byte quarters (quarter gq by one thread): FP32 A, real columns
// 16p..16p+15 (complex column 8p+w is the pair 2w, 2w+1); split FP64 A
// (QMC_PREC_FP32_SPLIT), real columns 8p..8p+7 as doubles (complex column
// 8p+w carries hi and lo of real column 8p+w).  Columns at or beyond t
// read as zero.
// ---------------------------------------------------------------------------
template <bool SPLIT>
__device__ __forceinline__ void stage_a_quarter(const PassArgs& a, bool a16, int j, int p, int gq, cx<float>* dst) {
  if constexpr (SPLIT) {
    const double* Ad = reinterpret_cast<const double*>(a.A);
    double* dd = reinterpret_cast<double*>(dst);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int col = 8 * p + 2 * gq + q;
      const int bytes = col < a.t ? 8 : 0;
      cp_async8_zfill(dd + q, bytes ? Ad + (int64_t)j * a.lda + col : Ad, bytes);
    }
  } else {
    const float* Af = reinterpret_cast<const float*>(a.A);
    const int col0 = 16 * p + 4 * gq;
    if (a16) {
      int bytes = (a.t - col0) * 4;
      bytes = bytes < 0 ? 0 : (bytes > 16 ? 16 : bytes);
      cp_async16_zfill(dst, bytes ? Af + (int64_t)j * a.lda + col0 : Af, bytes);
    } else {  // rows not 16-byte aligned (odd t): four 4-byte copies
      float* dstf = reinterpret_cast<float*>(dst);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int bytes = col0 + q < a.t ? 4 : 0;
        cp_async4_zfill(dstf + q, bytes ? Af + (int64_t)j * a.lda + col0 + q : Af, bytes);
      }
    }
  }
}

// The complex value of a staged piece (unscaled): FP32 A as is; split FP64
// A as (hi, lo) = (fp32(x), fp32(x - hi)).
template <bool SPLIT>
__device__ __forceinline__ cx<float> staged_value(const cx<float>& raw) {
  if constexpr (SPLIT) {
    const double x = *reinterpret_cast<const double*>(&raw);
    const float hi = (float)x;
    return mk<float>(hi, (float)(x - (double)hi));
  } else {
    return raw;
  }
}

// Column scales of complex column c: FP32 pairs (2c, 2c+1); split (c, c).
template <bool SPLIT>
__device__ __forceinline__ void column_scales(const PassArgs& a, int c, float& s0, float& s1) {
  if constexpr (SPLIT) {
    s0 = s1 = c < a.t ? __ldg(a.cscale + c) : 0.f;
  } else {
    const int c2 = 2 * c;
    s0 = c2 < a.t ? __ldg(a.cscale + c2) : 0.f;
    s1 = c2 + 1 < a.t ? __ldg(a.cscale + c2 + 1) : 0.f;
  }
}

// ---------------------------------------------------------------------------
// First pass: scatter-add from the padded gather table, forward P x Q
// transform, twiddle w_L^{-n2·k1}.  Lines with at most kDirectEntries
// entries take their DFT term by term instead.
// ---------------------------------------------------------------------------
template <int P, int Q, bool SPLIT>
__global__ void __launch_bounds__(PqPipeShape<P, Q>::NT, PqPipeShape<P, Q>::MINB) k_pqpipe_gather(const __grid_constant__ PassArgs a,
                                                                        int ntiles) {
  auto first_of = [&]() -> int { return (int)blockIdx.x; };
  auto step_of = [&]() -> int { return (int)gridDim.x; };
#include "qmc_pqpipe_gather_body.inc"
}

// ---------------------------------------------------------------------------
// First pass, lines with at most kDirectEntries entries (the plan lists
// them): each line's DFT summed term by term, X_i = Σ_e v_e·w_LP^{-n_e·i},
// then the twiddle w_L^{-n2·i}.  Without the transform's registers and
// shared tile this kernel keeps four blocks per SM and all threads busy:
// thread (g, w) forms the points i = g + 32·k of column w.  Entries and
// twiddles of the next tile are copied with cp.async while this one sums.
// ---------------------------------------------------------------------------
template <int LP>
struct PqDirectShape {
  static constexpr int NT = 256;
  static constexpr int KO = LP / 32;                       // points per thread
  static constexpr int STG = kDirectEntries * kLines;      // staged A segments (complex)
  static constexpr int SLOT = ((STG + LP + kDirectEntries + 1) / 2) * 2;
};

template <int LP, bool SPLIT>
__global__ void __launch_bounds__(256, 4) k_pq_direct(const __grid_constant__ PassArgs a, int ntiles) {
  auto first_of = [&]() -> int { return (int)blockIdx.x; };
  auto step_of = [&]() -> int { return (int)gridDim.x; };
  auto direct_lines = [&]() -> int { return a.n_direct; };
  auto direct_line = [&](int v) -> int { return __ldg(a.lines + a.n_pair + v); };
#include "qmc_pq_direct_body.inc"
}

}  // namespace
}  // namespace qmc
