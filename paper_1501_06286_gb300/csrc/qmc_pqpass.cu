// qmc_pqpass.cu — register-resident kernels for the single-transform passes
// (pass A: scatter-add + forward transform; pass C: inverse transform +
// un-permute; and their adjoint counterparts) when the pass length is a
// product LP = P·Q of two different small factors: 768 = 24·32,
// 255 = 15·17, 80 = 16·5, 96 = 12·8, 128 = 16·8, 160 = 16·10.
//
// Point i = q + Q·p.  Stage 1: thread q (q < Q) holds x[q + Q·p] for all p,
// does a P-point DFT over p, multiplies by w_LP^{q·k_p} and writes the
// values transposed into shared memory.  Stage 2: thread k_p (k_p < P)
// reads its Q values and does a Q-point DFT over q, ending with
// X[k_p + P·k_q] for all k_q.  A line uses max(P, Q) threads; the ones past
// Q (stage 1) or past P (stage 2) wait.  P- and Q-point DFTs are built from
// the radix codelets of fft_engine.cuh: fixed 2, 3, 4, 5, 8, 16, 32 and,
// for a product N = A·B of those, one level of the same decomposition with
// twiddles from the block's table.
#include "qmc_io.cuh"

namespace qmc {

namespace {

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

}  // namespace

enum PqMode : int { PQ_FWD = 0, PQ_INV = 2 };

template <int P, int Q>
struct PqShape {
  static constexpr int TPL = P > Q ? P : Q;                // threads per line
  static constexpr int NT = ((TPL * kLines + 31) / 32) * 32;  // whole warps
};

template <int P, int Q, int LOAD, int STORE, int MODE>
__global__ void __launch_bounds__(PqShape<P, Q>::NT)
    k_pq(const __grid_constant__ PassArgs a) {
  constexpr int LP = P * Q;
  constexpr int R = P > Q ? P : Q;  // register array length
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* S = tw + LP;
  const int tid = threadIdx.x;
  const int w = tid & 7, tl = tid >> 3;  // column, thread-in-line
  const int p = blockIdx.y;
  const int ag = blockIdx.x;             // one line group per block (8 columns)
  const int c = (p << 3) + w;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += blockDim.x) tw[k] = twL[(int64_t)k * tstep];
  }
  const int64_t rbase = (int64_t)ag * a.line_stride;
  const int64_t pstride = a.point_stride;
  cx<float> x[R];
#pragma unroll
  for (int k = 0; k < R; ++k) x[k] = mk<float>(0.f, 0.f);
  // ---- stage-1 input: points tl + Q*p ------------------------------------
  if constexpr (LOAD == LD_GATHER_A) {
    gather_tile<float>(a, S, (LP + LP / Q) * kLines, ag, 1, 3, p,
                       [=](int i, int, int ww) { return qidx<Q>(i, ww); });
    if (tl < Q) {
#pragma unroll
      for (int k = 0; k < P; ++k) x[k] = S[qidx<Q>(tl + Q * k, w)];
    }
    __syncthreads();
  } else {
    if (tl < Q) {
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int64_t r = rbase + (int64_t)(tl + Q * k) * pstride;
        if constexpr (LOAD == LD_SCRATCH)
          x[k] = reinterpret_cast<const cx<float>*>(a.scratch)[((int64_t)p * a.L + r) * 8 + w];
        else
          x[k] = load_input<float, LOAD>(a, r, c);
      }
    }
    __syncthreads();  // twiddle table ready
  }
  // Output rows of the line's points (un-permute pass), loaded into shared
  // memory before the transform so that their latency overlaps it and the
  // stores below do not wait on them one by one; the transform's first
  // barrier publishes them.
  const bool act = tl < P;
  int* rows = reinterpret_cast<int*>(S + (LP + LP / Q) * kLines);
  if constexpr (STORE == ST_OUT) {
    for (int i = tid; i < LP; i += blockDim.x) rows[i] = __ldg(a.orow + rbase + (int64_t)i * pstride);
  }
  pq_fft<P, Q, MODE == PQ_FWD ? -1 : +1>(x, S, tw, tl, w);

  // ---- output: points tl + P*k (threads tl < P) --------------------------
  float esum = 0.f;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int i = tl + P * k;
    const int64_t r = rbase + (int64_t)i * pstride;
    cx<float> val = x[k];
    if (act && a.twiddle) {
      const cx<float> wv = twL[(int64_t)ag * i];
      val = a.twiddle > 0 ? twmul<+1>(val, wv) : twmul<-1>(val, wv);
    }
    if constexpr (STORE == ST_SCRATCH) {
      if (act) reinterpret_cast<cx<float>*>(a.scratch)[((int64_t)p * a.L + r) * 8 + w] = val;
    } else if constexpr (STORE == ST_OUT) {
      float contrib = 0.f;
      int64_t row = -1;
      if (act && c < a.T) {
        row = rows[i];
        contrib = store_out_row<float>(a, row, c, val, esum);
      }
      if (a.row_mean) row_mean_add(a, contrib, row, w, 8);
    } else if constexpr (STORE == ST_DA) {
      if (act && c < a.T) store_da<float>(a, r, c, val);
    }
  }
  if constexpr (STORE == ST_OUT) {
    if (a.exp_sum) exp_sum_flush(a, esum);
  }
}

template <int P, int Q, int LOAD, int STORE, int MODE>
static int run_pq(const PassArgs& a, cudaStream_t st) {
  constexpr int LP = P * Q;
  const size_t smem = sizeof(cx<float>) * ((size_t)LP + (size_t)(LP + LP / Q) * kLines) +
                      (STORE == ST_OUT ? sizeof(int) * (size_t)LP : 0);
  static size_t configured = 48 * 1024;
  if (smem > configured) {
    if (cudaFuncSetAttribute(k_pq<P, Q, LOAD, STORE, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return QMC_ERR_UNSUPPORTED;
    }
    configured = smem;
  }
  dim3 grid(a.n_linegroups, (a.T + 7) >> 3);
  k_pq<P, Q, LOAD, STORE, MODE><<<grid, PqShape<P, Q>::NT, smem, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int P, int Q>
static int dispatch_pq(const PassArgs& a, int load, int store, int mode, cudaStream_t st) {
  if (mode == PQ_FWD && load == LD_GATHER_A && store == ST_SCRATCH)
    return run_pq<P, Q, LD_GATHER_A, ST_SCRATCH, PQ_FWD>(a, st);
  if (mode == PQ_FWD && load == LD_PERM_G && store == ST_SCRATCH)
    return run_pq<P, Q, LD_PERM_G, ST_SCRATCH, PQ_FWD>(a, st);
  if (mode == PQ_INV && load == LD_SCRATCH && store == ST_OUT)
    return run_pq<P, Q, LD_SCRATCH, ST_OUT, PQ_INV>(a, st);
  if (mode == PQ_INV && load == LD_SCRATCH && store == ST_DA)
    return run_pq<P, Q, LD_SCRATCH, ST_DA, PQ_INV>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

bool pq_pass_supported(int LP) {
  return LP == 768 || LP == 255 || LP == 80 || LP == 96 || LP == 128 || LP == 160;
}

// Single-transform passes (pass A / pass C and their adjoints) with 8-column
// panels; QMC_ERR_UNSUPPORTED for anything else.
int launch_pq_pass(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (a.logW != 3 || (a.fwd && a.inv)) return QMC_ERR_UNSUPPORTED;
  const int mode = a.fwd ? PQ_FWD : PQ_INV;
  switch (a.LP) {
    case 768: return dispatch_pq<24, 32>(a, load, store, mode, st);
    case 255: return dispatch_pq<15, 17>(a, load, store, mode, st);
    case 80: return dispatch_pq<16, 5>(a, load, store, mode, st);
    case 96: return dispatch_pq<12, 8>(a, load, store, mode, st);
    case 128: return dispatch_pq<16, 8>(a, load, store, mode, st);
    case 160: return dispatch_pq<16, 10>(a, load, store, mode, st);
  }
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
