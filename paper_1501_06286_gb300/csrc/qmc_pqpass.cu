// qmc_pqpass.cu — register-resident kernels for the single-transform passes
// (pass A: scatter-add + forward transform; pass C: inverse transform +
// un-permute; and their adjoint counterparts) when the pass length is a
// product LP = P·Q of two different small factors: 768 = 24·32,
// 255 = 15·17, 50 = 10·5, 80 = 16·5, 96 = 12·8, 128 = 16·8, 160 = 16·10.  One block
// per line of 8 columns; the transform is in qmc_pq.cuh.  A line uses
// max(P, Q) threads; the ones past Q (stage 1) or past P (stage 2) wait.
#include "qmc_io.cuh"
#include "qmc_pq.cuh"

namespace qmc {

using namespace pq;

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
  // one line of one 8-column panel per block, panels fastest: the panels
  // of a line write neighbouring pieces of the same output rows at about
  // the same time (whole sectors for rows that are not 16-byte multiples)
  const int p = blockIdx.x;
  const int ag = blockIdx.y;
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
    for (int i = tid; i < LP; i += blockDim.x) rows[i] = chk(__ldg(a.orow + rbase + (int64_t)i * pstride), a.n_out, a.err);
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
  static KernelSetup setup;
  if (const int rc = setup_kernel(k_pq<P, Q, LOAD, STORE, MODE>, setup, smem, PqShape<P, Q>::NT, nullptr))
    return rc;
  dim3 grid((a.T + 7) >> 3, a.n_linegroups);
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
  if (mode == PQ_FWD && load == LD_SCRATCH && store == ST_SCRATCH)  // after a dense scatter-add
    return run_pq<P, Q, LD_SCRATCH, ST_SCRATCH, PQ_FWD>(a, st);
  if (mode == PQ_INV && load == LD_SCRATCH && store == ST_OUT)
    return run_pq<P, Q, LD_SCRATCH, ST_OUT, PQ_INV>(a, st);
  if (mode == PQ_INV && load == LD_SCRATCH && store == ST_DA)
    return run_pq<P, Q, LD_SCRATCH, ST_DA, PQ_INV>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

bool pq_pass_supported(int LP) {
  return LP == 768 || LP == 255 || LP == 50 || LP == 80 || LP == 96 || LP == 128 || LP == 160;
}

// Single-transform passes (pass A / pass C and their adjoints) with 8-column
// panels; QMC_ERR_UNSUPPORTED for anything else.
int launch_pq_pass(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (a.logW != 3 || (a.fwd && a.inv)) return QMC_ERR_UNSUPPORTED;
  const int mode = a.fwd ? PQ_FWD : PQ_INV;
  switch (a.LP) {
    case 768: return dispatch_pq<24, 32>(a, load, store, mode, st);
    case 255: return dispatch_pq<15, 17>(a, load, store, mode, st);
    case 50: return dispatch_pq<10, 5>(a, load, store, mode, st);
    case 80: return dispatch_pq<16, 5>(a, load, store, mode, st);
    case 96: return dispatch_pq<12, 8>(a, load, store, mode, st);
    case 128: return dispatch_pq<16, 8>(a, load, store, mode, st);
    case 160: return dispatch_pq<16, 10>(a, load, store, mode, st);
  }
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
