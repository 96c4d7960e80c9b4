// qmc_pq.cuh — transforms of length LP = P·Q (two different small factors)
// for one line of 8 complex columns held in registers, shared by the
// P x Q pass kernels (qmc_pqpass.cu, qmc_pqpipe.cu).
//
// Point i = q + Q·p.  Stage 1: thread q (q < Q) holds x[q + Q·p] for all p,
// does a P-point DFT over p, multiplies by w_LP^{q·k_p} and writes the
// values transposed into shared memory.  Stage 2: thread k_p (k_p < P)
// reads its Q values and does a Q-point DFT over q, ending with
// X[k_p + P·k_q] for all k_q.  P- and Q-point DFTs are built from the radix
// codelets of fft_engine.cuh: fixed 2, 3, 4, 5, 8, 16 and small primes,
// and for a product N = A·B of those, one level of the same decomposition
// with twiddles from the block's table.
#pragma once

#include "fft_engine.cuh"

namespace qmc {
namespace pq {

template <int N>
struct SplitOf {  // N = A * B: A the smallest odd prime factor, or 2 (or 4 for 32)
  static constexpr int A = (N % 3 == 0) ? 3 : (N % 5 == 0) ? 5 : (N == 32) ? 4 : 2;
  static constexpr int B = N / A;
};

template <int DIR, int N>
__device__ __forceinline__ void dftN(cx<float>* v, const cx<float>* tw, int LP);

// N = A·B (DIT): n = q + A·m; B-point DFTs over m, twiddle w_N^{q·k1},
// A-point DFTs over q; X[k1 + B·k2].
template <int DIR, int A, int B>
__device__ __forceinline__ void dft_composite(cx<float>* v, const cx<float>* tw, int LP) {
  constexpr int N = A * B;
  cx<float> y[A][B];
#pragma unroll
  for (int q = 0; q < A; ++q) {
#pragma unroll
    for (int m = 0; m < B; ++m) y[q][m] = v[q + A * m];
    dftN<DIR, B>(y[q], tw, LP);
  }
  const int step = LP / N;
#pragma unroll
  for (int q = 1; q < A; ++q) {
#pragma unroll
    for (int k1 = 1; k1 < B; ++k1) y[q][k1] = twmul<DIR>(y[q][k1], tw[q * k1 * step]);
  }
#pragma unroll
  for (int k1 = 0; k1 < B; ++k1) {
    cx<float> z[A];
#pragma unroll
    for (int q = 0; q < A; ++q) z[q] = y[q][k1];
    dftN<DIR, A>(z, tw, LP);
#pragma unroll
    for (int k2 = 0; k2 < A; ++k2) v[k1 + B * k2] = z[k2];
  }
}

template <int DIR, int N>
__device__ __forceinline__ void dftN(cx<float>* v, const cx<float>* tw, int LP) {
  if constexpr (N == 1) {
  } else if constexpr (N == 2) {
    dft2<DIR>(v[0], v[1]);
  } else if constexpr (N == 3) {
    dft3<DIR>(v);
  } else if constexpr (N == 4) {
    dft4<DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (N == 5) {
    dft5<DIR>(v);
  } else if constexpr (N == 8) {
    dft8<DIR>(v);
  } else if constexpr (N == 16) {
    dft16<DIR>(v);
  } else if constexpr (N == 7 || N == 11 || N == 13 || N == 17) {
    dft_prime<DIR, N>(v, tw, LP / N);
  } else {
    dft_composite<DIR, SplitOf<N>::A, SplitOf<N>::B>(v, tw, LP);
  }
}

constexpr int kLines = 8;  // 8 complex columns (one panel) per block

template <int Q>
__device__ __forceinline__ int qidx(int i, int w) { return (i + i / Q) * kLines + w; }

// LP = P·Q transform of one line: in x[q + Q·p] at v[p] for thread q < Q,
// out X[k_p + P·k_q] at v[k_q] for thread k_p < P.  All threads call it.
template <int P, int Q, int DIR>
__device__ __forceinline__ void pq_fft(cx<float>* v, cx<float>* S, const cx<float>* tw, int tl, int w) {
  constexpr int LP = P * Q;
  if (tl < Q) {
    dftN<DIR, P>(v, tw, LP);
#pragma unroll
    for (int k = 1; k < P; ++k) v[k] = twmul<DIR>(v[k], tw[tl * k]);
#pragma unroll
    for (int k = 0; k < P; ++k) S[qidx<Q>(k * Q + tl, w)] = v[k];
  }
  __syncthreads();
  if (tl < P) {
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = S[qidx<Q>(tl * Q + q, w)];
    dftN<DIR, Q>(v, tw, LP);
  }
  __syncthreads();
}

// Inverse LP = P·Q transform in the reverse order of pq_fft: on entry thread
// k_p (< P) holds Y[k_p + P·k_q] at v[k_q] (the output layout of pq_fft), on
// exit thread q (< Q) holds x[q + Q·p] = Σ_k Y[k] w_LP^{+(q + Q·p)·k} at v[p]
// (the input layout of pq_fft).  Since (q + Qp)(k_p + Pk_q) ≡ q·k_p +
// P·q·k_q + Q·p·k_p (mod PQ): a Q-point inverse DFT over k_q, the twiddle
// w_LP^{q·k_p}, a transpose, a P-point inverse DFT over k_p.
template <int P, int Q>
__device__ __forceinline__ void pq_ifft_rev(cx<float>* v, cx<float>* S, const cx<float>* tw, int tl, int w) {
  constexpr int LP = P * Q;
  if (tl < P) {
    dftN<+1, Q>(v, tw, LP);
#pragma unroll
    for (int q = 1; q < Q; ++q) v[q] = twmul<+1>(v[q], tw[q * tl]);
#pragma unroll
    for (int q = 0; q < Q; ++q) S[qidx<Q>(q + Q * tl, w)] = v[q];
  }
  __syncthreads();
  if (tl < Q) {
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = S[qidx<Q>(tl + Q * k, w)];
    dftN<+1, P>(v, tw, LP);
  }
  __syncthreads();
}

// Constants of a P x Q transform held in registers for the whole kernel
// (tl is fixed per thread): the stage-1 twiddles w_LP^{tl·k}, k = 1..P-1,
// and, when Q is an odd prime >= 7, its roots w_Q^m, m = 1..(Q-1)/2.
template <int P, int Q>
struct PqRegs {
  static constexpr bool kPrimeQ = Q == 7 || Q == 11 || Q == 13 || Q == 17;
  static constexpr int H = (Q - 1) / 2;
  cx<float> mid[P];
  cx<float> root[kPrimeQ ? H + 1 : 1];
  __device__ __forceinline__ void load(const cx<float>* tw, int tl) {
    constexpr int LP = P * Q;
#pragma unroll
    for (int k = 1; k < P; ++k) mid[k] = tw[(tl * k) % LP];
    if constexpr (kPrimeQ) {
#pragma unroll
      for (int m = 1; m <= H; ++m) root[m] = tw[m * (LP / Q)];
    }
  }
};

// Odd prime Q-point DFT by the symmetric direct sum (as dft_prime) with the
// roots from registers: w_Q^{idx} = root[idx] for idx <= H, else the
// conjugate of root[Q - idx]; the indices are constants once unrolled.
template <int DIR, int N, int PP>
__device__ __forceinline__ void dft_prime_regs(cx<float>* v, const PqRegs<PP, N>& rg) {
  constexpr int H = (N - 1) / 2;
  cx<float> sp[H], sm[H];
#pragma unroll
  for (int m = 1; m <= H; ++m) { sp[m - 1] = v[m] + v[N - m]; sm[m - 1] = v[m] - v[N - m]; }
  const cx<float> x0 = v[0];
  cx<float> s0 = x0;
#pragma unroll
  for (int m = 0; m < H; ++m) s0 = s0 + sp[m];
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    cx<float> re = x0, im = mk<float>(0.f, 0.f);
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      const int idx = (m * k) % N;
      const float wr = idx <= H ? rg.root[idx].re : rg.root[N - idx].re;
      const float wi = idx <= H ? rg.root[idx].im : -rg.root[N - idx].im;
      re = re + scale(sp[m - 1], wr);
      im = im + scale(sm[m - 1], wi);
    }
    const cx<float> d = muli<DIR>(im);
    v[k] = re + d;
    v[N - k] = re - d;
  }
  v[0] = s0;
}

// pq_fft with the constants of PqRegs.
template <int P, int Q, int DIR>
__device__ __forceinline__ void pq_fft(cx<float>* v, cx<float>* S, const cx<float>* tw, const PqRegs<P, Q>& rg,
                                       int tl, int w) {
  constexpr int LP = P * Q;
  if (tl < Q) {
    dftN<DIR, P>(v, tw, LP);
#pragma unroll
    for (int k = 1; k < P; ++k) v[k] = twmul<DIR>(v[k], rg.mid[k]);
#pragma unroll
    for (int k = 0; k < P; ++k) S[qidx<Q>(k * Q + tl, w)] = v[k];
  }
  __syncthreads();
  if (tl < P) {
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = S[qidx<Q>(tl * Q + q, w)];
    if constexpr (PqRegs<P, Q>::kPrimeQ) dft_prime_regs<DIR, Q>(v, rg);
    else dftN<DIR, Q>(v, tw, LP);
  }
  __syncthreads();
}

}  // namespace pq
}  // namespace qmc
