// qmc_io.cuh — element loads and stores at the two ends of the product,
// shared by every pass kernel.
//
//   load_input  (first pass)  forward: a'_r = Σ_{e_j = r} A_j (the
//               scatter-add P·a of Section 2.1), column-scaled;
//               adjoint: g'_r = G[out_row(r)] (or exp(B)/(rows·t)).
//   store_out   (last pass, forward): out[out_row(r)] = value / scale,
//               with the row-mean and exp-sum epilogues.
//   store_da    (last pass, adjoint): dA[j] = value / scale + φ(0)·G_0 for
//               every j with e_j = r (colliding j receive the same row).
#pragma once

#include "qmc_internal.h"

namespace qmc {

// Work-array loads bypass L1 (ld.global.cg): in the persistent batch kernel
// a block can read lines that another block of the same launch wrote.
__device__ __forceinline__ cx<float> ld_cg(const cx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}
__device__ __forceinline__ cx<double> ld_cg(const cx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}

template <typename R>
__device__ __forceinline__ cx<R> load_pair_f32(const float* row, int c2, int t, int vec2) {
  if (vec2 && c2 + 1 < t) {
    const float2 v = *reinterpret_cast<const float2*>(row + c2);
    return mk<R>(R(v.x), R(v.y));
  }
  const R re = c2 < t ? R(row[c2]) : R(0);
  const R im = c2 + 1 < t ? R(row[c2 + 1]) : R(0);
  return mk<R>(re, im);
}

template <typename R, int LOAD>
__device__ __forceinline__ cx<R> load_input(const PassArgs& a, int64_t r, int c) {
  cx<R> val = mk<R>(R(0), R(0));
  if constexpr (LOAD == LD_GATHER_A) {
    if (c < a.T) {
      const int beg = a.row_ptr[r], end = a.row_ptr[r + 1];
      R re = R(0), im = R(0);
      for (int q = beg; q < end; ++q) {
        const int64_t j = chk((int64_t)a.jlist[q], a.s_a, a.err);
        if (a.split) {
          const double x = reinterpret_cast<const double*>(a.A)[j * a.lda + c];
          const float hi = (float)x;
          re += R(hi);
          im += R((float)(x - (double)hi));
        } else if (a.a_f64) {
          const double* row = reinterpret_cast<const double*>(a.A) + j * a.lda;
          if (2 * c < a.t) re += R((float)row[2 * c]);
          if (2 * c + 1 < a.t) im += R((float)row[2 * c + 1]);
        } else {
          const float* row = reinterpret_cast<const float*>(a.A) + j * a.lda;
          const cx<R> z = load_pair_f32<R>(row, 2 * c, a.t, a.a_vec2);
          re += z.re;
          im += z.im;
        }
      }
      if (a.split) {
        const R sc = R(a.cscale[c]);
        val = mk<R>(re * sc, im * sc);
      } else {
        val = mk<R>(2 * c < a.t ? re * R(a.cscale[2 * c]) : R(0),
                    2 * c + 1 < a.t ? im * R(a.cscale[2 * c + 1]) : R(0));
      }
    }
  } else if constexpr (LOAD == LD_PERM_G) {
    if (c < a.T) {
      const int64_t row = chk((int64_t)a.orow[r], a.n_out, a.err);
      val = load_pair_f32<R>(a.G + row * a.ldg, 2 * c, a.t, a.g_vec2);
      if (a.g_exp) {
        val.re = (2 * c < a.t) ? R(expf((float)val.re) * a.g_scale) : R(0);
        val.im = (2 * c + 1 < a.t) ? R(expf((float)val.im) * a.g_scale) : R(0);
      }
      val.re = 2 * c < a.t ? val.re * R(a.cscale[2 * c]) : R(0);
      val.im = 2 * c + 1 < a.t ? val.im * R(a.cscale[2 * c + 1]) : R(0);
    }
  } else if constexpr (LOAD == LD_DENSE64) {
    if (c == 0) val = mk<R>(R(a.zeta[r]), R(0));
  } else if constexpr (LOAD == LD_PSET) {
    // Section 2.2: block b of the right-hand sides uses e_{b,j} = j·b mod L
    // (0-based j), so position u collects the j with j·b ≡ u (mod L): none
    // unless d = gcd(b, L) divides u, else j ≡ (u/d)·(b/d)^{-1} mod (L/d).
    R part[2] = {R(0), R(0)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = 2 * c + h;
      if (c < a.T && q < a.t) {
        const int b = q / a.t_a, k = q - b * a.t_a;
        const int d = a.ps_d[b];
        if (r % d == 0) {
          const int64_t Ld = a.L / d;
          int64_t j = ((r / d) * (int64_t)a.ps_inv[b]) % Ld;
          R acc = R(0);
          if (a.a_f64) {
            const double* col = reinterpret_cast<const double*>(a.A) + k;
            for (; j < a.s_a; j += Ld) acc += R((float)col[j * a.lda]);
          } else {
            const float* col = reinterpret_cast<const float*>(a.A) + k;
            for (; j < a.s_a; j += Ld) acc += R(col[j * a.lda]);
          }
          part[h] = acc * R(a.cscale[k]);
        }
      }
    }
    val = mk<R>(part[0], part[1]);
  }
  return val;
}

// First pass of the forward product: fills a zeroed shared tile with the
// scatter-add a'_u for the non-empty positions u of the tile's lines only
// (the plan lists them per first-pass line), so that a tile's global reads
// are the A rows it needs and nothing else.  idx(i, v, w) gives the tile
// slot of point i, line group v, column w.  Every thread of the block calls
// this; it ends with a barrier.
template <typename R, typename Idx, typename TM = BlockTeam>
__device__ __forceinline__ void gather_tile(const PassArgs& a, cx<R>* tile, int tile_elems, int ag0,
                                            int V, int logW, int p, Idx idx, const TM& tm = TM()) {
  const int W = 1 << logW;
  for (int e = tm.tid(); e < tile_elems; e += tm.nt()) tile[e] = mk<R>(R(0), R(0));
  tm.sync();
  for (int v = 0; v < V; ++v) {
    const int ag = ag0 + v;
    if (ag >= a.n_linegroups) break;
    const int b0 = a.bucket_ptr[ag], n = (a.bucket_ptr[ag + 1] - b0) << logW;
    for (int k = tm.tid(); k < n; k += tm.nt()) {
      const int w = k & (W - 1);
      const int u = chk(a.blist[b0 + (k >> logW)], (int64_t)a.L, a.err);
      const int i = chk((int)(((int64_t)u - (int64_t)ag * a.line_stride) / a.point_stride), (int64_t)a.LP, a.err);
      tile[idx(i, v, w)] = load_input<R, LD_GATHER_A>(a, u, (p << logW) + w);
    }
  }
  tm.sync();
}

// Forward product output.  Returns this element's contribution to the row
// sum (for the row-mean epilogue) and sets *row to its output row.
// The affine epilogue of qmc_matmul_affine: col_off[k] + b, then exp().
__device__ __forceinline__ float affine_out(const PassArgs& a, int k, float b) {
  if (a.col_off) b += a.col_off[k];
  return a.out_exp ? expf(b) : b;
}

template <typename R>
__device__ __forceinline__ float store_out_row(const PassArgs& a, int64_t row, int c, cx<R> val,
                                               float& esum) {
  float* orow_ptr = a.out + row * a.ldo;
  if (a.split) {
    float b = ((float)val.re + (float)val.im) * a.cinv[c];
    if (a.col_off || a.out_exp) b = affine_out(a, c, b);
    orow_ptr[c] = b;
    if (a.exp_sum) esum += expf(b);
    return b;
  }
  const int c2 = 2 * c;
  // generic loads: the scales may be in shared memory (qmc_small.cu)
  float re = (float)val.re * a.cinv[c2];
  float im = c2 + 1 < a.t ? (float)val.im * a.cinv[c2 + 1] : 0.f;
  if (a.col_off || a.out_exp) {
    re = affine_out(a, c2, re);
    if (c2 + 1 < a.t) im = affine_out(a, c2 + 1, im);
  }
  if (a.o_vec2 && c2 + 1 < a.t) {
    *reinterpret_cast<float2*>(orow_ptr + c2) = make_float2(re, im);
  } else {
    orow_ptr[c2] = re;
    if (c2 + 1 < a.t) orow_ptr[c2 + 1] = im;
  }
  if (a.exp_sum) esum += expf(re) + (c2 + 1 < a.t ? expf(im) : 0.f);
  return re + im;
}

template <typename R>
__device__ __forceinline__ float store_out(const PassArgs& a, int64_t r, int c, cx<R> val,
                                           float& esum, int64_t* row_out) {
  const int64_t row = chk((int64_t)__ldg(a.orow + r), a.n_out, a.err);
  *row_out = row;
  return store_out_row<R>(a, row, c, val, esum);
}

template <typename R>
__device__ __forceinline__ void store_da(const PassArgs& a, int64_t r, int c, cx<R> val) {
  const int beg = __ldg(a.row_ptr + r), end = __ldg(a.row_ptr + r + 1);
  if (beg >= end) return;
  const int c2 = 2 * c;
  val.re = val.re * R(a.cinv[c2]);
  val.im = c2 + 1 < a.t ? val.im * R(a.cinv[c2 + 1]) : R(0);
  if (a.has_row0) {
    cx<R> g0 = load_pair_f32<R>(a.G + (int64_t)a.row0_out * a.ldg, c2, a.t, a.g_vec2);
    if (a.g_exp) {
      g0.re = (c2 < a.t) ? R(expf((float)g0.re) * a.g_scale) : R(0);
      g0.im = (c2 + 1 < a.t) ? R(expf((float)g0.im) * a.g_scale) : R(0);
    }
    val = val + scale(g0, R(a.phi0));
  }
  const float re = (float)val.re, im = (float)val.im;
  for (int q = beg; q < end; ++q) {
    float* drow = a.dA + chk((int64_t)__ldg(a.jlist + q), a.s_a, a.err) * a.ldda;
    if (a.d_vec2 && c2 + 1 < a.t) {
      *reinterpret_cast<float2*>(drow + c2) = make_float2(re, im);
    } else {
      drow[c2] = re;
      if (c2 + 1 < a.t) drow[c2 + 1] = im;
    }
  }
}

// p-set output: real column q of the combined problem is column q % t_a of
// block b = q / t_a, whose rows start at ps_blk[b]·L.
template <typename R>
__device__ __forceinline__ void store_pset(const PassArgs& a, int64_t r, int c, cx<R> val) {
  const int64_t row = chk((int64_t)a.orow[r], (int64_t)a.L, a.err);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = 2 * c + h;
    if (q < a.t) {
      const int b = q / a.t_a, k = q - b * a.t_a;
      float v = (float)(h ? val.im : val.re) * a.cinv[k];
      if (a.col_off || a.out_exp) v = affine_out(a, k, v);
      a.out[((int64_t)a.ps_blk[b] * a.L + row) * a.ldo + k] = v;
    }
  }
}

// Sum over the W consecutive lanes that share an output row, then one
// atomic per row (row-mean epilogue).  All lanes of the warp must call it.
__device__ __forceinline__ void row_mean_add(const PassArgs& a, float contrib, int64_t row, int w, int W) {
  for (int off = W >> 1; off > 0; off >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, off);
  if (w == 0 && row >= 0) atomicAdd(a.row_mean + row, contrib * a.inv_t);
}

// Block reduction of the exp-sum partials (FP32 per thread, a few dozen
// terms each; FP64 from the warp sums on), one atomic per block.
__device__ __forceinline__ void exp_sum_flush(const PassArgs& a, float esum_f) {
  __shared__ double red[32];
  double esum = (double)esum_f;
  for (int off = 16; off > 0; off >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = esum;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (threadIdx.x == 0) atomicAdd(a.exp_sum, x);
  }
}

}  // namespace qmc
