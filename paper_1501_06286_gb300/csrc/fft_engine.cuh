// fft_engine.cuh — batched mixed-radix Stockham FFT on a tile held in
// shared memory (sm_103a).
//
// The product Z·a' of Section 2.1 (Eq. (3)) is evaluated "using FFT"; this
// file holds the transform.  A tile is LP points x M lines, element
// (point i, line m) at buf[i*M + m]; lines are independent columns (FFT
// batch), consecutive lines are consecutive addresses so that a warp's
// accesses are contiguous.  Each radix-r stage reads one buffer and writes
// the other in Stockham (self-sorting) order, so the result is in natural
// order with no bit reversal.
//
// Twiddles come from a table tw[k] = exp(+2 pi i k / LP), k < LP, filled
// from FP64 sin/cos rounded once (never generated by recurrence).  DIR = -1
// is the forward transform X_k = sum_n x_n e^{-2 pi i n k / LP}, DIR = +1
// the unnormalised inverse.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qmc {

template <typename R>
struct __align__(2 * sizeof(R)) cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> z; z.re = a; z.im = b; return z; }
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__device__ __forceinline__ cx<R> scale(cx<R> a, R s) { return mk<R>(a.re * s, a.im * s); }
template <typename R>
__device__ __forceinline__ cx<R> conj(cx<R> a) { return mk<R>(a.re, -a.im); }
// a * w when DIR = +1, a * conj(w) when DIR = -1 (w = exp(+i theta))
template <int DIR, typename R>
__device__ __forceinline__ cx<R> twmul(cx<R> a, cx<R> w) {
  if (DIR > 0) return a * w;
  return mk<R>(a.re * w.re + a.im * w.im, a.im * w.re - a.re * w.im);
}
// multiply by DIR * i
template <int DIR, typename R>
__device__ __forceinline__ cx<R> muli(cx<R> a) {
  return DIR > 0 ? mk<R>(-a.im, a.re) : mk<R>(a.im, -a.re);
}

// ---------------------------------------------------------------------------
// Radix-r DFT codelets on registers.  v[k] <- sum_n v[n] w_r^{DIR n k}.
// Constants are the exact values cos/sin of the listed angles.
// ---------------------------------------------------------------------------
template <int DIR, typename R>
__device__ __forceinline__ void dft2(cx<R>& a, cx<R>& b) {
  cx<R> t = a - b; a = a + b; b = t;
}

template <int DIR, typename R>
__device__ __forceinline__ void dft4(cx<R>& a0, cx<R>& a1, cx<R>& a2, cx<R>& a3) {
  cx<R> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = muli<DIR>(a1 - a3);
  a0 = t0 + t2; a2 = t0 - t2; a1 = t1 + t3; a3 = t1 - t3;
}

template <int DIR, typename R>
__device__ __forceinline__ void dft3(cx<R>* v) {
  const R h = R(0.86602540378443864676);   // sin(pi/3)
  cx<R> t = v[1] + v[2];
  cx<R> d = muli<DIR>(scale(v[1] - v[2], h));
  cx<R> m = v[0] - scale(t, R(0.5));
  v[0] = v[0] + t;
  v[1] = m + d;
  v[2] = m - d;
}

template <int DIR, typename R>
__device__ __forceinline__ void dft5(cx<R>* v) {
  const R c1 = R(0.30901699437494742410);   // cos(2pi/5)
  const R c2 = R(-0.80901699437494742410);  // cos(4pi/5)
  const R s1 = R(0.95105651629515357212);   // sin(2pi/5)
  const R s2 = R(0.58778525229247312917);   // sin(4pi/5)
  cx<R> t1 = v[1] + v[4], t2 = v[2] + v[3];
  cx<R> d1 = v[1] - v[4], d2 = v[2] - v[3];
  cx<R> a = v[0] + scale(t1, c1) + scale(t2, c2);
  cx<R> b = v[0] + scale(t1, c2) + scale(t2, c1);
  cx<R> p = muli<DIR>(scale(d1, s1) + scale(d2, s2));
  cx<R> q = muli<DIR>(scale(d1, s2) - scale(d2, s1));
  v[0] = v[0] + t1 + t2;
  v[1] = a + p; v[4] = a - p;
  v[2] = b + q; v[3] = b - q;
}

template <int DIR, typename R>
__device__ __forceinline__ void dft8(cx<R>* v) {
  const R c = R(0.70710678118654752440);    // cos(pi/4)
  // decimation in time: even / odd halves
  cx<R> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cx<R> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  // o_k *= w8^{DIR k}
  o1 = mk<R>(c * (o1.re - DIR * o1.im), c * (o1.im + DIR * o1.re));
  o2 = muli<DIR>(o2);
  o3 = mk<R>(-c * (o3.re + DIR * o3.im), c * (DIR * o3.re - o3.im));
  v[0] = e0 + o0; v[4] = e0 - o0;
  v[1] = e1 + o1; v[5] = e1 - o1;
  v[2] = e2 + o2; v[6] = e2 - o2;
  v[3] = e3 + o3; v[7] = e3 - o3;
}

template <int DIR, typename R>
__device__ __forceinline__ void dft16(cx<R>* v) {
  const R c8 = R(0.92387953251128675613);   // cos(pi/8)
  const R s8 = R(0.38268343236508977173);   // sin(pi/8)
  const R c4 = R(0.70710678118654752440);   // cos(pi/4)
  // n = q + 4 m: inner DFT4 over m for each q
  cx<R> y[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    y[q][0] = v[q]; y[q][1] = v[q + 4]; y[q][2] = v[q + 8]; y[q][3] = v[q + 12];
    dft4<DIR>(y[q][0], y[q][1], y[q][2], y[q][3]);
  }
  // twiddle y[q][k1] by w16^{DIR q k1}; w16^e = (cos(2 pi e/16), DIR sin(...))
  const R cs[10] = {R(1), c8, c4, s8, R(0), -s8, -c4, -c8, R(-1), -c8};
  const R sn[10] = {R(0), s8, c4, c8, R(1), c8, c4, s8, R(0), -s8};
#pragma unroll
  for (int q = 1; q < 4; ++q) {
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) {
      const int e = q * k1;
      cx<R> a = y[q][k1];
      if (e == 4) {          // w16^4 = i: a swap and a sign, no arithmetic
        y[q][k1] = muli<DIR>(a);
      } else if (e == 2 || e == 6) {  // c4·(±1 ± i): two adds, two multiplies
        const R sr = e == 2 ? R(1) : R(-1);
        const R u = a.re * sr - R(DIR) * a.im, v = a.im * sr + R(DIR) * a.re;
        y[q][k1] = mk<R>(c4 * u, c4 * v);
      } else {
        const R wr = cs[e], wi = R(DIR) * sn[e];
        y[q][k1] = mk<R>(a.re * wr - a.im * wi, a.re * wi + a.im * wr);
      }
    }
  }
  // outer DFT4 over q: X[k1 + 4 k2]
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cx<R> a0 = y[0][k1], a1 = y[1][k1], a2 = y[2][k1], a3 = y[3][k1];
    dft4<DIR>(a0, a1, a2, a3);
    v[k1] = a0; v[k1 + 4] = a1; v[k1 + 8] = a2; v[k1 + 12] = a3;
  }
}

// Odd prime radix P by the symmetric direct sum; w_P^m taken from the
// tile's twiddle table: tw[m * step] = exp(+2 pi i m / P).
template <int DIR, int P, typename R>
__device__ __forceinline__ void dft_prime(cx<R>* v, const cx<R>* tw, int step) {
  constexpr int H = (P - 1) / 2;
  cx<R> sp[H], sm[H];
#pragma unroll
  for (int m = 1; m <= H; ++m) { sp[m - 1] = v[m] + v[P - m]; sm[m - 1] = v[m] - v[P - m]; }
  cx<R> x0 = v[0];
  cx<R> s0 = x0;
#pragma unroll
  for (int m = 0; m < H; ++m) s0 = s0 + sp[m];
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    cx<R> re = x0, im = mk<R>(R(0), R(0));
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      const cx<R> w = tw[((m * k) % P) * step];
      re = re + scale(sp[m - 1], w.re);
      im = im + scale(sm[m - 1], w.im);
    }
    cx<R> d = muli<DIR>(im);
    v[k] = re + d;
    v[P - k] = re - d;
  }
  v[0] = s0;
}

template <int DIR, int RAD, typename R>
__device__ __forceinline__ void butterfly(cx<R>* v, const cx<R>* tw, int LP) {
  if constexpr (RAD == 2) dft2<DIR>(v[0], v[1]);
  else if constexpr (RAD == 3) dft3<DIR>(v);
  else if constexpr (RAD == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
  else if constexpr (RAD == 5) dft5<DIR>(v);
  else if constexpr (RAD == 8) dft8<DIR>(v);
  else if constexpr (RAD == 16) dft16<DIR>(v);
  else dft_prime<DIR, RAD>(v, tw, LP / RAD);
}

// Nominal elements per thread: the host launches NT >= LP*M/kEPT threads.
constexpr int kEPT = 16;
constexpr int kMaxStages = 8;

// The threads that work on one tile and their barrier: the whole block
// (every stand-alone kernel), or a part of it with a named barrier of its
// own (the batch queue runs two generic tiles per block, one per half).
struct BlockTeam {
  static constexpr bool kWhole = true;
  __device__ __forceinline__ int tid() const { return (int)threadIdx.x; }
  __device__ __forceinline__ int nt() const { return (int)blockDim.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// One Stockham radix-RAD stage over an LP x M tile, out of place
// (src -> dst), one butterfly per loop iteration.
//   ns: product of the radices of the earlier stages.
template <int DIR, int RAD, typename R, typename TM>
__device__ __forceinline__ void fft_stage(const cx<R>* __restrict__ src, cx<R>* __restrict__ dst,
                                          const cx<R>* tw, int LP, int logM, int ns, const TM& tm) {
  const int M = 1 << logM;
  const int nb = LP / RAD;
  const int items = nb << logM;
  const int step = LP / (ns * RAD);
  for (int it = tm.tid(); it < items; it += tm.nt()) {
    const int m = it & (M - 1), b = it >> logM;
    const int j = b % ns;
    cx<R> v[RAD];
#pragma unroll
    for (int k = 0; k < RAD; ++k) v[k] = src[((b + k * nb) << logM) + m];
    if (ns > 1) {
#pragma unroll
      for (int k = 1; k < RAD; ++k) v[k] = twmul<DIR>(v[k], tw[j * k * step]);
    }
    butterfly<DIR, RAD>(v, tw, LP);
    const int idx = (b - j) * RAD + j;
#pragma unroll
    for (int k = 0; k < RAD; ++k) dst[((idx + k * ns) << logM) + m] = v[k];
  }
  tm.sync();
}

// Stage radices packed 5 bits each (stage st's radix is (bits >> 5*st) & 31)
// so that the stage loop reads them from a register, not local memory.
struct Radices {
  int n;
  int r[kMaxStages];
  __host__ __device__ uint64_t packed() const {
    uint64_t b = 0;
    for (int i = 0; i < n; ++i) b |= (uint64_t)r[i] << (5 * i);
    return b;
  }
};

// Stage code of a length-257 transform done by Rader's algorithm.
constexpr int kRader257 = 31;

// Tables of Rader's algorithm for p = 257 with primitive root 3:
//   pin[a]  = 3^a mod 257,  pout[b] = 3^{-b} mod 257   (a, b < 256)
//   what[k] = DFT_256(w)_k / 256,  w_m = exp(DIR 2 pi i 3^{-m} / 257)
//   tw256   = exp(+2 pi i k / 256) in shared memory
// With u_a = x[3^a]:  X[0] = x_0 + sum_a u_a and
// X[3^{-b}] = x_0 + (u (*) w)_b, a 256-point cyclic convolution done with
// two 256-point FFTs; the same primitive-root reordering that turns the
// lattice product into a circulant (Section 2.1) turns a prime-length DFT
// into a cyclic convolution.
template <typename R>
struct RaderRefs {
  const cx<R>* tw256;      // shared memory
  const cx<R>* what_fwd;   // global
  const cx<R>* what_inv;   // global
  const int16_t* pin;      // global
  const int16_t* pout;     // global
  cx<R>* x0s;              // shared memory, M entries
  cx<R>* u0s;              // shared memory, M entries
};

template <int DIR, typename R, typename TM>
__device__ __forceinline__ cx<R>* fft_stages(cx<R>* buf, cx<R>* alt, const cx<R>* tw, int LP,
                                             int logM, int nst, uint64_t rbits, const TM& tm);

template <int DIR, typename R, typename TM>
__device__ __forceinline__ cx<R>* rader257(cx<R>* buf, cx<R>* alt, int logM, const RaderRefs<R>& rr,
                                           const TM& tm) {
  const int M = 1 << logM;
  const int n = 256 << logM;
  for (int it = tm.tid(); it < n; it += tm.nt()) {
    const int m = it & (M - 1), q = it >> logM;
    alt[it] = buf[((int)rr.pin[q] << logM) + m];
  }
  for (int m = tm.tid(); m < M; m += tm.nt()) rr.x0s[m] = buf[m];
  tm.sync();
  const uint64_t r16 = 16u | (16u << 5);
  cx<R>* U = fft_stages<-1, R>(alt, buf, rr.tw256, 256, logM, 2, r16, tm);
  const cx<R>* what = DIR < 0 ? rr.what_fwd : rr.what_inv;
  for (int it = tm.tid(); it < n; it += tm.nt()) {
    const int m = it & (M - 1), k = it >> logM;
    if (k == 0) rr.u0s[m] = U[it];
    U[it] = U[it] * what[k];
  }
  tm.sync();
  cx<R>* other = U == alt ? buf : alt;
  cx<R>* Cv = fft_stages<+1, R>(U, other, rr.tw256, 256, logM, 2, r16, tm);
  cx<R>* dst = Cv == alt ? buf : alt;
  for (int it = tm.tid(); it < n; it += tm.nt()) {
    const int m = it & (M - 1), b = it >> logM;
    dst[((int)rr.pout[b] << logM) + m] = rr.x0s[m] + Cv[it];
  }
  for (int m = tm.tid(); m < M; m += tm.nt()) dst[m] = rr.x0s[m] + rr.u0s[m];
  tm.sync();
  return dst;
}

// Full LP-point transform of every line of the tile (natural order in and
// out), ping-ponging between buf and alt.  Returns the buffer holding the
// result.
template <int DIR, typename R, typename TM>
__device__ __forceinline__ cx<R>* fft_stages(cx<R>* buf, cx<R>* alt, const cx<R>* tw, int LP,
                                             int logM, int nst, uint64_t rbits, const TM& tm) {
  int ns = 1;
  cx<R>* src = buf;
  cx<R>* dst = alt;
  for (int st = 0; st < nst; ++st) {
    const int r = (int)((rbits >> (5 * st)) & 31u);
    switch (r) {
      case 2: fft_stage<DIR, 2>(src, dst, tw, LP, logM, ns, tm); break;
      case 3: fft_stage<DIR, 3>(src, dst, tw, LP, logM, ns, tm); break;
      case 4: fft_stage<DIR, 4>(src, dst, tw, LP, logM, ns, tm); break;
      case 5: fft_stage<DIR, 5>(src, dst, tw, LP, logM, ns, tm); break;
      case 7: fft_stage<DIR, 7>(src, dst, tw, LP, logM, ns, tm); break;
      case 8: fft_stage<DIR, 8>(src, dst, tw, LP, logM, ns, tm); break;
      case 11: fft_stage<DIR, 11>(src, dst, tw, LP, logM, ns, tm); break;
      case 13: fft_stage<DIR, 13>(src, dst, tw, LP, logM, ns, tm); break;
      case 16: fft_stage<DIR, 16>(src, dst, tw, LP, logM, ns, tm); break;
      case 17: fft_stage<DIR, 17>(src, dst, tw, LP, logM, ns, tm); break;
      default: break;  // rejected on the host
    }
    ns *= r;
    cx<R>* t = src; src = dst; dst = t;
  }
  return src;
}

template <int DIR, typename R, typename TM = BlockTeam>
__device__ __forceinline__ cx<R>* fft_tile(cx<R>* buf, cx<R>* alt, const cx<R>* tw, int LP,
                                           int logM, int nst, uint64_t rbits,
                                           const RaderRefs<R>& rr, const TM& tm = TM()) {
  if (nst == 1 && (int)(rbits & 31u) == kRader257) return rader257<DIR, R>(buf, alt, logM, rr, tm);
  return fft_stages<DIR, R>(buf, alt, tw, LP, logM, nst, rbits, tm);
}

}  // namespace qmc
