// qmc_pass_kernel.cuh — one pass of the fast product over the L x T work
// array (sm_103a).
//
// Section 2.1 computes Y'a = Z(Pa): a scatter-add P·a, a circulant product
// Z·a' "using FFT", then the rows are returned to the conventional order.
// With L = L1·L2 and row index r = n1·L2 + n2 the length-L transform is
// done as three passes (four-step FFT), each a batch of short FFTs on a
// shared-memory tile:
//   pass A  (points n1, lines n2):  load a' (scatter-add of A's rows),
//           forward FFT_L1, multiply by w_L^{-n2·k1};
//   pass B  (points n2, lines k1):  forward FFT_L2, multiply by the
//           spectrum H[k1 + L1·k2] (stored at row k1·L2 + k2), inverse
//           FFT_L2, multiply by w_L^{+n2·k1};
//   pass C  (points k1, lines n2):  inverse FFT_L1, write circulant row
//           r = n1·L2 + n2 to output row out_row(r).
// For L small enough a single pass does all of it (L2 = 1).  The same
// kernel, with other load/store modes, runs the adjoint and the plan-time
// FP64 spectrum.
#pragma once

#include "qmc_internal.h"

namespace qmc {

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

template <typename R, int LOAD, int STORE>
__global__ void __launch_bounds__(512) k_pass(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* buf = tw + a.LP;
  cx<R>* alt = buf + (a.LP << a.logM);
  RaderRefs<R> rr{};
  const bool rader = a.nst == 1 && (int)(a.rbits & 31u) == kRader257;
  if (rader) {
    cx<R>* t256 = alt + (a.LP << a.logM);
    const cx<R>* tab = reinterpret_cast<const cx<R>*>(a.rader);
    for (int k = threadIdx.x; k < 256; k += blockDim.x) t256[k] = tab[k];
    rr.tw256 = t256;
    rr.what_fwd = tab + 256;
    rr.what_inv = tab + 512;
    rr.pin = a.rader_perm;
    rr.pout = a.rader_perm + 256;
    rr.x0s = t256 + 256;
    rr.u0s = rr.x0s + (1 << a.logM);
  }
  const int LP = a.LP;
  const int W = 1 << a.logW, V = 1 << a.logV;
  const int p = blockIdx.y;
  const int a0 = blockIdx.x * V;
  const int tid = threadIdx.x, nt = blockDim.x;
  const cx<R>* twL = reinterpret_cast<const cx<R>*>(a.twL);
  const int tstep = a.L / LP;
  for (int k = tid; k < LP; k += nt) tw[k] = twL[(int64_t)k * tstep];

  const int items = LP << a.logM;
  // ---- load -------------------------------------------------------------
  for (int it = tid; it < items; it += nt) {
    const int w = it & (W - 1);
    const int v = (it >> a.logW) & (V - 1);
    const int i = it >> a.logM;
    const int ag = a0 + v;
    const int c = (p << a.logW) + w;
    cx<R> val = mk<R>(R(0), R(0));
    if (ag < a.n_linegroups) {
      const int64_t r = (int64_t)ag * a.line_stride + (int64_t)i * a.point_stride;
      if constexpr (LOAD == LD_SCRATCH) {
        val = reinterpret_cast<const cx<R>*>(a.scratch)[((int64_t)p * a.L + r) * W + w];
      } else if constexpr (LOAD == LD_GATHER_A) {
        if (c < a.T) {
          const int beg = a.row_ptr[r], end = a.row_ptr[r + 1];
          R re = R(0), im = R(0);
          for (int q = beg; q < end; ++q) {
            const int64_t j = a.jlist[q];
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
          const int64_t row = a.orow[r];
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
      }
    }
    buf[it] = val;
  }
  __syncthreads();

  // ---- transforms and spectral product ---------------------------------
  if (a.fwd) {
    cx<R>* res = fft_tile<-1>(buf, alt, tw, LP, a.logM, a.nst, a.rbits, rr);
    if (res != buf) { alt = buf; buf = res; }
  }
  if (a.mul) {
    const cx<R>* H = reinterpret_cast<const cx<R>*>(a.H);
    for (int it = tid; it < items; it += nt) {
      const int v = (it >> a.logW) & (V - 1);
      const int i = it >> a.logM;
      const int ag = a0 + v;
      if (ag < a.n_linegroups) {
        const int64_t r = (int64_t)ag * a.line_stride + (int64_t)i * a.point_stride;
        const cx<R> h = H[r];
        buf[it] = a.mul == 1 ? buf[it] * h : buf[it] * conj(h);
      }
    }
    __syncthreads();
  }
  if (a.inv) {
    cx<R>* res = fft_tile<+1>(buf, alt, tw, LP, a.logM, a.nst, a.rbits, rr);
    if (res != buf) { alt = buf; buf = res; }
  }

  // ---- store ------------------------------------------------------------
  double esum = 0.0;
  for (int base = 0; base < items; base += nt) {
    const int it = base + tid;
    const bool in_tile = it < items;
    const int w = it & (W - 1);
    const int v = (it >> a.logW) & (V - 1);
    const int i = it >> a.logM;
    const int ag = a0 + v;
    const int c = (p << a.logW) + w;
    const bool line_ok = in_tile && ag < a.n_linegroups;
    const int64_t r = (int64_t)ag * a.line_stride + (int64_t)i * a.point_stride;
    cx<R> val = in_tile ? buf[it] : mk<R>(R(0), R(0));
    if (line_ok && a.twiddle) {
      const cx<R> wv = twL[(int64_t)ag * i];
      val = a.twiddle > 0 ? twmul<+1>(val, wv) : twmul<-1>(val, wv);
    }
    if constexpr (STORE == ST_SCRATCH) {
      if (line_ok) reinterpret_cast<cx<R>*>(a.scratch)[((int64_t)p * a.L + r) * W + w] = val;
    } else if constexpr (STORE == ST_OUT) {
      float contrib = 0.f;
      int64_t row = -1;
      if (line_ok && c < a.T) {
        row = a.orow[r];
        float* orow_ptr = a.out + row * a.ldo;
        if (a.split) {
          const float b = ((float)val.re + (float)val.im) * a.cinv[c];
          orow_ptr[c] = b;
          contrib = b;
          if (a.exp_sum) esum += exp((double)b);
        } else {
          const int c2 = 2 * c;
          const float re = (float)val.re * a.cinv[c2];
          const float im = c2 + 1 < a.t ? (float)val.im * a.cinv[c2 + 1] : 0.f;
          if (a.o_vec2 && c2 + 1 < a.t) {
            *reinterpret_cast<float2*>(orow_ptr + c2) = make_float2(re, im);
          } else {
            orow_ptr[c2] = re;
            if (c2 + 1 < a.t) orow_ptr[c2 + 1] = im;
          }
          contrib = re + (c2 + 1 < a.t ? im : 0.f);
          if (a.exp_sum) esum += exp((double)re) + (c2 + 1 < a.t ? exp((double)im) : 0.0);
        }
      }
      if (a.row_mean) {
        // the W lanes sharing (i, v) are consecutive and W-aligned in the warp
        for (int off = W >> 1; off > 0; off >>= 1)
          contrib += __shfl_xor_sync(0xffffffffu, contrib, off);
        if (w == 0 && row >= 0) atomicAdd(a.row_mean + row, contrib * a.inv_t);
      }
    } else if constexpr (STORE == ST_DA) {
      if (line_ok && c < a.T) {
        const int beg = a.row_ptr[r], end = a.row_ptr[r + 1];
        if (beg < end) {
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
            float* drow = a.dA + (int64_t)a.jlist[q] * a.ldda;
            if (a.d_vec2 && c2 + 1 < a.t) {
              *reinterpret_cast<float2*>(drow + c2) = make_float2(re, im);
            } else {
              drow[c2] = re;
              if (c2 + 1 < a.t) drow[c2 + 1] = im;
            }
          }
        }
      }
    }
  }
  if constexpr (STORE == ST_OUT) {
    if (a.exp_sum) {
      // block reduction of the exp-sum partials, one atomic per block
      __shared__ double red[32];
      for (int off = 16; off > 0; off >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, off);
      __syncthreads();
      if ((tid & 31) == 0) red[tid >> 5] = esum;
      __syncthreads();
      if (tid < 32) {
        double x = tid < (nt >> 5) ? red[tid] : 0.0;
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (tid == 0) atomicAdd(a.exp_sum, x);
      }
    }
  }
}

}  // namespace qmc
