// qmc_pass_kernel.cuh — one pass of the fast product over the L x T work
// array (sm_103a), generic in the pass length.
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
// FP64 spectrum.  Lengths 256 and 1024 have a faster kernel
// (qmc_fastpass.cu); this one takes every length the radix set covers.
#pragma once

#include "qmc_io.cuh"

namespace qmc {

// One tile (line-group block bx, panel by) of a pass; every thread of the
// team (the block, by default) calls it.  k_pass runs one tile per block;
// the persistent batch kernel (qmc_batch.cu) runs many, one per half-block
// team at a time.
template <typename R, int LOAD, int STORE, typename TM = BlockTeam>
__device__ __forceinline__ void pass_tile(const PassArgs& a, int bx, int by, unsigned char* smem_raw,
                                          const TM& tm = TM()) {
  cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* buf = tw + a.LP;
  cx<R>* alt = buf + (a.LP << a.logM);
  RaderRefs<R> rr{};
  const bool rader = a.nst == 1 && (int)(a.rbits & 31u) == kRader257;
  if (rader) {
    cx<R>* t256 = alt + (a.LP << a.logM);
    const cx<R>* tab = reinterpret_cast<const cx<R>*>(a.rader);
    for (int k = tm.tid(); k < 256; k += tm.nt()) t256[k] = tab[k];
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
  const int p = by;
  const int a0 = bx * V;
  const int tid = tm.tid(), nt = tm.nt();
  const cx<R>* twL = reinterpret_cast<const cx<R>*>(a.twL);
  const int tstep = a.L / LP;
  for (int k = tid; k < LP; k += nt) tw[k] = twL[(int64_t)k * tstep];

  const int items = LP << a.logM;
  // ---- load -------------------------------------------------------------
  if constexpr (LOAD == LD_GATHER_A) {
    const int logW = a.logW, logM = a.logM;
    gather_tile<R>(a, buf, items, a0, V, logW, p,
                   [=](int i, int v, int w) { return (i << logM) + (v << logW) + w; }, tm);
  } else {
  for (int it = tid; it < items; it += nt) {
    const int w = it & (W - 1);
    const int v = (it >> a.logW) & (V - 1);
    const int i = it >> a.logM;
    const int ag = a0 + v;
    const int c = (p << a.logW) + w;
    cx<R> val = mk<R>(R(0), R(0));
    if (ag < a.n_linegroups) {
      const int64_t r = (int64_t)ag * a.line_stride + (int64_t)i * a.point_stride;
      if constexpr (LOAD == LD_SCRATCH)
        val = ld_cg(reinterpret_cast<const cx<R>*>(a.scratch) + ((int64_t)p * a.L + r) * W + w);
      else
        val = load_input<R, LOAD>(a, r, c);
    }
    buf[it] = val;
  }
  tm.sync();
  }

  // ---- transforms and spectral product ---------------------------------
  if (a.fwd) {
    cx<R>* res = fft_tile<-1>(buf, alt, tw, LP, a.logM, a.nst, a.rbits, rr, tm);
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
    tm.sync();
  }
  if (a.inv) {
    cx<R>* res = fft_tile<+1>(buf, alt, tw, LP, a.logM, a.nst, a.rbits, rr, tm);
    if (res != buf) { alt = buf; buf = res; }
  }

  // ---- store ------------------------------------------------------------
  float esum = 0.f;
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
      if (line_ok && c < a.T) contrib = store_out<R>(a, r, c, val, esum, &row);
      if (a.row_mean) row_mean_add(a, contrib, row, w, W);
    } else if constexpr (STORE == ST_DA) {
      if (line_ok && c < a.T) store_da<R>(a, r, c, val);
    } else if constexpr (STORE == ST_PSET) {
      if (line_ok && c < a.T) store_pset<R>(a, r, c, val);
    }
  }
  if constexpr (STORE == ST_OUT && TM::kWhole) {
    if (a.exp_sum) exp_sum_flush(a, esum);  // block reduction (the queue's items have no epilogues)
  }
}

template <typename R, int LOAD, int STORE>
__global__ void __launch_bounds__(512) k_pass(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_tile<R, LOAD, STORE>(a, blockIdx.x, blockIdx.y, smem_raw);
}

}  // namespace qmc
