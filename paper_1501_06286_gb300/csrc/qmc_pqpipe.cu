// qmc_pqpipe.cu — persistent, double-buffered versions of the P x Q pass
// kernels (pass lengths LP = P·Q: 768 = 24·32, 255 = 15·17, 50 = 10·5) for the two
// single-transform passes of the forward product and the adjoint's
// permuted gather:
//   * the un-permute pass (inverse transform over k1, output rows
//     out_row(r), FP32 store, with the exp-sum epilogue when asked; the
//     plain store of the 768-point pass runs two panels per tile);
//   * the first pass (scatter-add of A's rows from the padded gather
//     table, forward transform over n1, twiddle w_L^{-n2·k1}).
// Each block loops over tiles (one line of one 8-column panel).  The
// un-permute pass copies tile i+1 (64-byte point segments, with the line's
// output rows) into the other shared buffer with cp.async while it
// transforms tile i; the first pass stages the next tile's A segments and
// twiddles the same way.  The transform is the one of qmc_pq.cuh.
#include "qmc_pqpipe.cuh"

namespace qmc {

using namespace pq;

namespace {

// Pairs of neighbouring term-by-term lines (2λ, 2λ+1) in one tile: point i
// of the two lines sits in neighbouring rows of the work array, so every
// point leaves as one 128-byte write (the single-line kernel writes 64-byte
// pieces at a stride of L2 rows, which the memory takes at a lower rate).
// Thread (g, line, w): 16 lanes per point group, 512 threads.
template <int LP>
struct PqDirect2Shape {
  static constexpr int NT = 512;
  static constexpr int KO = LP / 32;
  static constexpr int STG = 2 * kDirectEntries * kLines;
  static constexpr int SLOT = ((STG + 2 * LP + 2 * kDirectEntries + 1) / 2) * 2;
};

template <int LP, bool SPLIT>
__global__ void __launch_bounds__(512, 2) k_pq_direct2(const __grid_constant__ PassArgs a, int ntiles) {
  using S_ = PqDirect2Shape<LP>;
  constexpr int NT = S_::NT, KO = S_::KO, STG = S_::STG, SLOT = S_::SLOT, E = kDirectEntries;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* slots = tw + ((LP + 1) / 2) * 2;
  const int tid = threadIdx.x;
  const int w16 = tid & 15, sub = w16 >> 3, w = w16 & 7, g = tid >> 4;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += NT) tw[k] = twL[(int64_t)k * tstep];
  }
  __syncthreads();
  const int em = a.gp_em;
  const int nl = a.n_pair;
  const int ge = tid >> 2, gq = tid & 3;  // prefetch role (tid < 8·E): entry of both lines, 16-byte quarter
  const int gl = ge / E, gee = ge % E;

  const bool a16 = (a.lda % 4) == 0 && ((reinterpret_cast<uintptr_t>(a.A) & 15u) == 0);
  const int64_t pst = (int64_t)a.point_stride * kLines;

  auto prefetch = [&](int tile, cx<float>* slot) {
    const int ag0 = __ldg(a.lines + tile % nl), p = tile / nl;
    cx<float>* stg = slot;
    cx<float>* twl = slot + STG;
    int* idx = reinterpret_cast<int*>(twl + 2 * LP);
    if (ge < 2 * E) {
      int i = -1, j = 0;
      if (gee < em) {
        i = __ldg(a.gp_i + (ag0 + gl) * em + gee);
        j = __ldg(a.gp_j + (ag0 + gl) * em + gee);
        if (i >= 0) {
          i = chk(i, (int64_t)LP, a.err);
          j = chk(j, a.s_a, a.err);
        }
      }
      if (gq == 0) idx[ge] = i;
      if (i >= 0) {
        stage_a_quarter<SPLIT>(a, a16, j, p, gq, stg + ge * kLines + 2 * gq);
      }
    }
    for (int k = tid; k < 2 * LP; k += NT) {
      const int l = k >= LP ? 1 : 0, kk = k - l * LP;
      cp_async8(twl + k, twL + (int64_t)(ag0 + l) * kk);
    }
    cp_async_commit();
  };

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, slots);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    cx<float>* cur = slots + (it & 1) * SLOT;
    cx<float>* nxt = slots + ((it + 1) & 1) * SLOT;
    const int next = tile + gridDim.x;
    if (next < ntiles) prefetch(next, nxt);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const int ag0 = __ldg(a.lines + tile % nl), p = tile / nl;
    const cx<float>* stg = cur;
    const cx<float>* twl = cur + STG;
    const int* idx = reinterpret_cast<const int*>(twl + 2 * LP);
    float s0, s1;
    column_scales<SPLIT>(a, (p << 3) + w, s0, s1);

    cx<float> x[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) x[k] = mk<float>(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = idx[sub * E + e];
      if (n < 0) break;  // padding (point -1) comes last
      const cx<float> v0 = staged_value<SPLIT>(stg[(sub * E + e) * kLines + w]);
      const cx<float> v = mk<float>(v0.re * s0, v0.im * s1);
      int m = (n * g) % LP;   // n·i mod LP, stepped by n·32 along k
      const int d = (n * 32) % LP;
#pragma unroll
      for (int k = 0; k < KO; ++k) {
        x[k] = x[k] + twmul<-1>(v, tw[m]);
        m += d;
        m -= m >= LP ? LP : 0;
      }
    }
    cx<float>* obase = reinterpret_cast<cx<float>*>(a.scratch) +
                       ((int64_t)p * a.L + (int64_t)(ag0 + sub) * a.line_stride) * kLines + w;
#pragma unroll
    for (int k = 0; k < KO; ++k) {
      const int i = g + 32 * k;
      obase[i * pst] = twmul<-1>(x[k], twl[sub * LP + i]);
    }
    __syncthreads();  // the next iteration's prefetch overwrites this slot
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Adjoint first pass: g'_r = G[out_row(r)] (or exp(B)·scale), forward P x Q
// transform, twiddle w_L^{-n2·k1}.  The rows of G a tile needs are known
// only after its output-row indices arrive, so the indices are loaded two
// tiles ahead and the G pieces one tile ahead, both into registers.  Tiles
// run panel fastest: the panels of one line read neighbouring pieces of
// the same rows of G together.
// ---------------------------------------------------------------------------
template <int P, int Q>
__global__ void __launch_bounds__(PqPipeShape<P, Q>::NT, (P * Q >= 512 ? 1 : 3)) k_pqpipe_permg(const __grid_constant__ PassArgs a,
                                                                         int ntiles) {
  using S_ = PqPipeShape<P, Q>;
  constexpr int LP = S_::LP, NT = S_::NT;
  constexpr int R = P > Q ? P : Q;
  constexpr bool kRegs = P * Q < 512;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* S = tw + ((LP + 1) / 2) * 2;
  const int tid = threadIdx.x;
  const int w = tid & 7, tl = tid >> 3;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += NT) tw[k] = twL[(int64_t)k * tstep];
  }
  __syncthreads();
  PqRegs<P, Q> rg;  // register constants (short lines only, for the budget)
  if constexpr (kRegs) rg.load(tw, tl);
  const int npan = (a.T + 7) >> 3;
  const int64_t pstride = a.point_stride;
  const bool loader = tl < Q;

  auto load_rows = [&](int tile, int* rows) {
    if (tile < ntiles && loader) {
      const int* src = a.orow + (int64_t)(tile / npan) * a.line_stride + tl * pstride;
#pragma unroll
      for (int k = 0; k < P; ++k) rows[k] = chk(__ldg(src + (int64_t)Q * k * pstride), a.n_out, a.err);
    }
  };
  auto load_g = [&](int tile, const int* rows, float2* g) {
    if (tile < ntiles && loader) {
      const int c2 = 2 * (((tile % npan) << 3) + w);
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const float* row = a.G + (int64_t)rows[k] * a.ldg;
        if (a.g_vec2 && c2 + 1 < a.t) {
          g[k] = __ldg(reinterpret_cast<const float2*>(row + c2));
        } else {
          g[k].x = c2 < a.t ? __ldg(row + c2) : 0.f;
          g[k].y = c2 + 1 < a.t ? __ldg(row + c2 + 1) : 0.f;
        }
      }
    }
  };

  int rows_n[P];
  float2 g_n[P];
#pragma unroll
  for (int k = 0; k < P; ++k) { rows_n[k] = 0; g_n[k] = make_float2(0.f, 0.f); }
  int tile = blockIdx.x;
  load_rows(tile, rows_n);
  load_g(tile, rows_n, g_n);
  load_rows(tile + gridDim.x, rows_n);
  __syncthreads();  // twiddle table
  for (; tile < ntiles; tile += gridDim.x) {
    const int ag = tile / npan, p = tile % npan;
    const int c = (p << 3) + w, c2 = 2 * c;
    cx<float> x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = mk<float>(0.f, 0.f);
    if (loader && c < a.T) {  // this tile's G pieces, loaded one tile ago
      const float s0 = __ldg(a.cscale + c2), s1 = c2 + 1 < a.t ? __ldg(a.cscale + c2 + 1) : 0.f;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        float re = g_n[k].x, im = g_n[k].y;
        if (a.g_exp) {
          re = c2 < a.t ? expf(re) * a.g_scale : 0.f;
          im = c2 + 1 < a.t ? expf(im) * a.g_scale : 0.f;
        }
        x[k] = mk<float>(re * s0, im * s1);
      }
    }
    const int next = tile + gridDim.x;
    load_g(next, rows_n, g_n);                 // G pieces of the next tile
    load_rows(next + gridDim.x, rows_n);       // row indices of the one after
    if constexpr (kRegs) pq_fft<P, Q, -1>(x, S, tw, rg, tl, w);
    else pq_fft<P, Q, -1>(x, S, tw, tl, w);
    if (tl < P) {
      cx<float>* obase = reinterpret_cast<cx<float>*>(a.scratch) +
                         ((int64_t)p * a.L + (int64_t)ag * a.line_stride) * kLines + w;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const int i = tl + P * k;
        const float2 wv = __ldg(reinterpret_cast<const float2*>(twL) + (int64_t)ag * i);
        obase[(int64_t)i * pstride * kLines] = twmul<-1>(x[k], mk<float>(wv.x, wv.y));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Spectral pass of a four-step product for short inner lengths LP = P·Q:
// forward transform (pq_fft), × H (MUL 1) or × conj(H) (MUL 2), inverse
// transform in the reverse order (pq_ifft_rev, which returns the points to
// the layout they were loaded in), twiddle w_L^{+ag·i}, store.  Points are
// contiguous rows; the tile, its spectrum entries and its twiddles are
// copied with cp.async one tile ahead.
// ---------------------------------------------------------------------------
template <int P, int Q, int MUL>
__global__ void __launch_bounds__(PqPipeShape<P, Q>::NT) k_pqpipe_spec(const __grid_constant__ PassArgs a,
                                                                     int ntiles) {
  using S_ = PqPipeShape<P, Q>;
  constexpr int LP = S_::LP, NT = S_::NT, SZ = S_::SZ;
  constexpr int SLOT = ((SZ + 2 * LP + 1) / 2) * 2;
  constexpr int R = P > Q ? P : Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* bufs = tw + ((LP + 1) / 2) * 2;
  const int tid = threadIdx.x;
  const int w = tid & 7, tl = tid >> 3;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += NT) tw[k] = twL[(int64_t)k * tstep];
  }
  const cx<float>* scratch_in = reinterpret_cast<const cx<float>*>(a.scratch);
  const cx<float>* H = reinterpret_cast<const cx<float>*>(a.H);
  const int nlg = a.n_linegroups;

  auto prefetch = [&](int tile, cx<float>* dst) {
    const int ag = tile % nlg, p = tile / nlg;
    const int64_t rb = (int64_t)ag * a.line_stride;
    const cx<float>* base = scratch_in + ((int64_t)p * a.L + rb) * kLines;
    for (int c = tid; c < LP * 4; c += NT) {  // 16-byte chunk: point c/4, columns 2*(c%4), +1
      const int i = c >> 2, part = (c & 3) * 2;
      cp_async16(dst + qidx<Q>(i, part), base + i * kLines + part);
    }
    cx<float>* hs = dst + SZ;
    cx<float>* ts = hs + LP;
    for (int k = tid; k < LP; k += NT) {
      cp_async8(hs + k, H + rb + k);
      cp_async8(ts + k, twL + (int64_t)ag * k);
    }
    cp_async_commit();
  };

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, bufs);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    cx<float>* cur = bufs + (it & 1) * SLOT;
    cx<float>* nxt = bufs + ((it + 1) & 1) * SLOT;
    const int next = tile + gridDim.x;
    if (next < ntiles) prefetch(next, nxt);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();  // this tile (and, first time round, the table) is in
    cx<float> x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = mk<float>(0.f, 0.f);
    if (tl < Q) {
#pragma unroll
      for (int k = 0; k < P; ++k) x[k] = cur[qidx<Q>(tl + Q * k, w)];
    }
    __syncthreads();
    pq_fft<P, Q, -1>(x, cur, tw, tl, w);
    const cx<float>* hs = cur + SZ;
    const cx<float>* ts = hs + LP;
    if (tl < P) {
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const cx<float> h = hs[tl + P * k];
        x[k] = MUL == 1 ? x[k] * h : x[k] * conj(h);
      }
    }
    pq_ifft_rev<P, Q>(x, cur, tw, tl, w);
    if (tl < Q) {
      const int ag = tile % nlg, p = tile / nlg;
      cx<float>* obase = reinterpret_cast<cx<float>*>(a.scratch) +
                         ((int64_t)p * a.L + (int64_t)ag * a.line_stride) * kLines + w;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int i = tl + Q * k;
        obase[i * kLines] = twmul<+1>(x[k], ts[i]);
      }
    }
    // the next iteration's prefetch overwrites this slot's spectrum and
    // twiddles, which the stores above have just read
    __syncthreads();
  }
  cp_async_wait<0>();
}

template <typename K>
int persistent_launch(K kernel, int nt, size_t smem, int ntiles, const PassArgs& a, cudaStream_t st,
                      KernelSetup& setup) {
  int grid = 0;
  if (const int rc = setup_kernel(kernel, setup, smem, nt, &grid)) return rc;
  if (grid > ntiles) grid = ntiles;
  kernel<<<grid, nt, smem, st>>>(a, ntiles);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int P, int Q, int KIND>
int run_out(const PassArgs& a, cudaStream_t st) {
  using S_ = PqPipeShape<P, Q>;
  static KernelSetup setup;
  const size_t smem = sizeof(cx<float>) * (((S_::LP + 1) / 2) * 2 +
                                           2 * (size_t)(KIND == 2 ? S_::DA_SLOT : S_::OUT_SLOT));
  const int ntiles = a.n_linegroups * ((a.T + 7) >> 3);
  return persistent_launch(k_pqpipe_out<P, Q, KIND>, S_::NT, smem, ntiles, a, st, setup);
}

template <int P, int Q, bool SPLIT>
int run_gather(const PassArgs& a, cudaStream_t st) {
  using S_ = PqPipeShape<P, Q>;
  static KernelSetup setup;
  const size_t smem =
      sizeof(cx<float>) * (((S_::LP + 1) / 2) * 2 + (size_t)S_::SZ + 2 * (size_t)S_::GATHER_SLOT);
  const int npan = (a.T + 7) >> 3;
  if constexpr ((P * Q) % 32 == 0) {
    if (a.lines) {
      // the plan's lines split by entry count: pairs of term-by-term lines,
      // single term-by-term lines, then the transform lines
      int rc = QMC_OK;
      if (a.n_pair > 0) {
        using D_ = PqDirect2Shape<P * Q>;
        static KernelSetup psetup;
        const size_t psmem = sizeof(cx<float>) * (((P * Q + 1) / 2) * 2 + 2 * (size_t)D_::SLOT);
        rc = persistent_launch(k_pq_direct2<P * Q, SPLIT>, D_::NT, psmem, a.n_pair * npan, a, st, psetup);
      }
      if (rc == QMC_OK && a.n_direct > 0) {
        using D_ = PqDirectShape<P * Q>;
        static KernelSetup dsetup;
        const size_t dsmem = sizeof(cx<float>) * (((P * Q + 1) / 2) * 2 + 2 * (size_t)D_::SLOT);
        rc = persistent_launch(k_pq_direct<P * Q, SPLIT>, D_::NT, dsmem, a.n_direct * npan, a, st, dsetup);
      }
      if (rc == QMC_OK && a.n_fft > 0)
        rc = persistent_launch(k_pqpipe_gather<P, Q, SPLIT>, S_::NT, smem, a.n_fft * npan, a, st, setup);
      return rc;
    }
  }
  PassArgs b = a;
  b.lines = nullptr;
  return persistent_launch(k_pqpipe_gather<P, Q, SPLIT>, S_::NT, smem, a.n_linegroups * npan, b, st, setup);
}

template <int P, int Q>
int run_permg(const PassArgs& a, cudaStream_t st) {
  using S_ = PqPipeShape<P, Q>;
  static KernelSetup setup;
  const size_t smem = sizeof(cx<float>) * (((S_::LP + 1) / 2) * 2 + (size_t)S_::SZ);
  const int ntiles = a.n_linegroups * ((a.T + 7) >> 3);
  return persistent_launch(k_pqpipe_permg<P, Q>, S_::NT, smem, ntiles, a, st, setup);
}

template <int P, int Q>
int run_spec(const PassArgs& a, cudaStream_t st) {
  using S_ = PqPipeShape<P, Q>;
  const size_t smem = sizeof(cx<float>) * (((S_::LP + 1) / 2) * 2 + 2 * (size_t)(((S_::SZ + 2 * S_::LP + 1) / 2) * 2));
  const int ntiles = a.n_linegroups * ((a.T + 7) >> 3);
  if (a.mul == 1) {
    static KernelSetup setup;
    return persistent_launch(k_pqpipe_spec<P, Q, 1>, S_::NT, smem, ntiles, a, st, setup);
  }
  static KernelSetup setup;
  return persistent_launch(k_pqpipe_spec<P, Q, 2>, S_::NT, smem, ntiles, a, st, setup);
}

// ---------------------------------------------------------------------------
// Un-permute pass over two panels per tile (16 complex columns, 512
// threads, one block per SM, double-buffered): each output row receives one
// 128-byte run per tile instead of two 64-byte runs from two tiles.  Rows
// of B scattered by the un-permute cost far more per byte in 64-byte pieces
// than in 128-byte ones, and more again when the row length is not a
// multiple of 16 bytes (odd t: every piece straddles sectors); measured on
// the field workload (t = 4225) this pass went from 10.9 to 8.8 ms.  Plain
// FP32 store (no epilogues); the two panels' points are read as two
// 64-byte segments each.
// ---------------------------------------------------------------------------
constexpr int kLines2 = 16;
template <int Q>
__device__ __forceinline__ int qidx2(int i, int w) { return (i + i / Q) * kLines2 + w; }

template <int P, int Q, int DIR>
__device__ __forceinline__ void pq_fft2(cx<float>* v, cx<float>* S, const cx<float>* tw, int tl, int w) {
  constexpr int LP = P * Q;
  if (tl < Q) {
    dftN<DIR, P>(v, tw, LP);
#pragma unroll
    for (int k = 1; k < P; ++k) v[k] = twmul<DIR>(v[k], tw[tl * k]);
#pragma unroll
    for (int k = 0; k < P; ++k) S[qidx2<Q>(k * Q + tl, w)] = v[k];
  }
  __syncthreads();
  if (tl < P) {
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = S[qidx2<Q>(tl * Q + q, w)];
    dftN<DIR, Q>(v, tw, LP);
  }
  __syncthreads();
}

template <int P, int Q>
struct PqPipe2Shape {
  static constexpr int LP = P * Q;
  static constexpr int TPL = P > Q ? P : Q;
  static constexpr int NT = TPL * kLines2;
  static constexpr int SZ = (LP + LP / Q) * kLines2;
  static constexpr int ROWS_CX = ((LP + 3) / 4) * 2;
  static constexpr int SLOT = SZ + ROWS_CX;
};

template <int P, int Q, bool SPLIT>
__global__ void __launch_bounds__(PqPipe2Shape<P, Q>::NT, 1) k_pqpipe_out2(const __grid_constant__ PassArgs a,
                                                                           int ntiles) {
  using S_ = PqPipe2Shape<P, Q>;
  constexpr int LP = S_::LP, NT = S_::NT, SZ = S_::SZ, SLOT = S_::SLOT;
  constexpr int R = P > Q ? P : Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* bufs = tw + ((LP + 1) / 2) * 2;
  const int tid = threadIdx.x;
  const int w = tid & 15, tl = tid >> 4;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += NT) tw[k] = twL[(int64_t)k * tstep];
  }
  __syncthreads();
  const cx<float>* scratch_in = reinterpret_cast<const cx<float>*>(a.scratch);
  const int64_t pst = (int64_t)a.point_stride * kLines;
  const int npan = (a.T + 7) >> 3;
  const int npair = (npan + 1) >> 1;

  auto prefetch = [&](int tile, cx<float>* dst) {
    const int ag = tile / npair, pp = tile % npair;
    const int64_t rb = (int64_t)ag * a.line_stride;
    const bool two = 2 * pp + 1 < npan;
    for (int c = tid; c < LP * 8; c += NT) {  // 16-byte chunk: point c/8, columns 2*(c%8), +1
      const int i = c >> 3, part = (c & 7) * 2;
      const int panel = 2 * pp + (part >> 3);
      cx<float>* d = dst + qidx2<Q>(i, part);
      if (part < 8 || two) {
        cp_async16(d, scratch_in + ((int64_t)panel * a.L + rb) * kLines + i * pst + (part & 7));
      } else {
        d[0] = mk<float>(0.f, 0.f);
        d[1] = mk<float>(0.f, 0.f);
      }
    }
    int* rows = reinterpret_cast<int*>(dst + SZ);
    for (int i = tid; i < LP; i += NT) cp_async4(rows + i, a.orow + rb + (int64_t)i * a.point_stride);
    cp_async_commit();
  };

  const bool o_vec2 = a.o_vec2 != 0;
  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, bufs);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    cx<float>* cur = bufs + (it & 1) * SLOT;
    cx<float>* nxt = bufs + ((it + 1) & 1) * SLOT;
    const int next = tile + gridDim.x;
    if (next < ntiles) prefetch(next, nxt);
    else cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    cx<float> x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = mk<float>(0.f, 0.f);
    if (tl < Q) {
#pragma unroll
      for (int k = 0; k < P; ++k) x[k] = cur[qidx2<Q>(tl + Q * k, w)];
    }
    __syncthreads();
    pq_fft2<P, Q, +1>(x, cur, tw, tl, w);

    const int pp = tile % npair;
    const int c = (pp << 4) + w;  // complex column
    const int* rows = reinterpret_cast<const int*>(cur + SZ);
    if constexpr (SPLIT) {
      // split precision: real column c is hi + lo of complex column c, so
      // the 16 lanes of a point write one 64-byte run of its row
      if (tl < P && c < a.T) {
        const float sc = __ldg(a.cinv + c);
        float* ocol = a.out + c;
#pragma unroll
        for (int k = 0; k < Q; ++k) ocol[chk((int64_t)rows[tl + P * k], a.n_out, a.err) * a.ldo] = (x[k].re + x[k].im) * sc;
      }
    } else if (!o_vec2) {
      // one 128-byte run per row: lane j of the warp writes real column
      // 32·pp + j of point tl0 + hh, fetched from lane 16·hh + j/2
      const int lane = tid & 31, j = lane;
      const int tl0 = tl & ~1;
      const int col = 32 * pp + j;
      const float sc = col < a.t ? __ldg(a.cinv + col) : 0.f;
      float* ocol = a.out + col;
#pragma unroll
      for (int k = 0; k < Q; ++k) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int src = 16 * hh + (j >> 1);
          const float re = __shfl_sync(0xffffffffu, x[k].re, src);
          const float im = __shfl_sync(0xffffffffu, x[k].im, src);
          if (tl0 + hh < P && col < a.t) ocol[chk((int64_t)rows[tl0 + hh + P * k], a.n_out, a.err) * a.ldo] = ((j & 1) ? im : re) * sc;
        }
      }
    } else if (tl < P && c < a.T) {
      const int c2 = 2 * c;
      const bool pair = c2 + 1 < a.t;
      const float s0 = __ldg(a.cinv + c2), s1 = pair ? __ldg(a.cinv + c2 + 1) : 0.f;
      float* ocol = a.out + c2;
      if (pair) {
#pragma unroll
        for (int k = 0; k < Q; ++k)
          *reinterpret_cast<float2*>(ocol + chk((int64_t)rows[tl + P * k], a.n_out, a.err) * a.ldo) = make_float2(x[k].re * s0, x[k].im * s1);
      } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) ocol[chk((int64_t)rows[tl + P * k], a.n_out, a.err) * a.ldo] = x[k].re * s0;
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

template <int P, int Q, bool SPLIT>
int run_out2(const PassArgs& a, cudaStream_t st) {
  using S_ = PqPipe2Shape<P, Q>;
  static KernelSetup setup;
  const size_t smem = sizeof(cx<float>) * (((S_::LP + 1) / 2) * 2 + 2 * (size_t)S_::SLOT);
  const int npair = (((a.T + 7) >> 3) + 1) >> 1;
  const int ntiles = a.n_linegroups * npair;
  return persistent_launch(k_pqpipe_out2<P, Q, SPLIT>, S_::NT, smem, ntiles, a, st, setup);
}

}  // namespace

// Spectral pass (LD_SCRATCH -> ST_SCRATCH, forward and inverse, × H or
// × conj(H), store twiddle +1, contiguous points) for inner lengths 80, 96,
// 128, 160; QMC_ERR_UNSUPPORTED otherwise.
int launch_pqpipe_spectral(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (a.logW != 3 || !(a.fwd && a.inv) || load != LD_SCRATCH || store != ST_SCRATCH || a.point_stride != 1 ||
      a.twiddle != 1 || (a.mul != 1 && a.mul != 2))
    return QMC_ERR_UNSUPPORTED;
  switch (a.LP) {
    case 80: return run_spec<10, 8>(a, st);
    case 96: return run_spec<12, 8>(a, st);
    case 128: return run_spec<16, 8>(a, st);
    case 160: return run_spec<16, 10>(a, st);
  }
  return QMC_ERR_UNSUPPORTED;
}

// Persistent P x Q passes: the un-permute pass (LD_SCRATCH -> ST_OUT,
// inverse, no twiddle, no split columns, no fused row mean; with or without
// the exp-sum epilogue), the adjoint's last pass (LD_SCRATCH -> ST_DA), the
// first pass from
// the padded gather table (FP32 A; 16-byte copies when its rows are 16-byte
// aligned, 4-byte copies otherwise) and the adjoint's first pass
// (LD_PERM_G -> ST_SCRATCH).
// Anything else is QMC_ERR_UNSUPPORTED.
int launch_pqpipe_pass(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (a.logW != 3 || (a.fwd && a.inv) || a.mul) return QMC_ERR_UNSUPPORTED;
  const bool out = load == LD_SCRATCH && store == ST_OUT && !a.fwd && a.twiddle == 0 && !a.split &&
                   !a.row_mean && !a.col_off && !a.out_exp;
  // split precision (FP64 A as hi + lo): the 768-point first pass and the
  // plain two-panel un-permute pass
  const bool out_split = load == LD_SCRATCH && store == ST_OUT && !a.fwd && a.twiddle == 0 && a.split &&
                         !a.row_mean && !a.col_off && !a.out_exp && !a.exp_sum && a.LP == 768;
  const bool gather_split = load == LD_GATHER_A && store == ST_SCRATCH && a.fwd && a.twiddle < 0 &&
                            a.gp_em >= 1 && a.gp_em <= kGatherMax && a.a_f64 && a.split && a.LP == 768 &&
                            (((uintptr_t)a.A) & 7u) == 0;
  if (out_split) return run_out2<24, 32, true>(a, st);
  if (gather_split) return run_gather<24, 32, true>(a, st);
  const bool esum = a.exp_sum != nullptr;
  const bool da = load == LD_SCRATCH && store == ST_DA && !a.fwd && a.twiddle == 0 && !a.split;
  const int kind = da ? 2 : esum ? 1 : 0;
  const bool gather = load == LD_GATHER_A && store == ST_SCRATCH && a.fwd && a.twiddle < 0 && a.gp_em >= 1 &&
                      a.gp_em <= kGatherMax && !a.a_f64 && !a.split && (((uintptr_t)a.A) & 3u) == 0;
  const bool permg = load == LD_PERM_G && store == ST_SCRATCH && a.fwd && a.twiddle < 0;
  if (!out && !gather && !permg && !da) return QMC_ERR_UNSUPPORTED;
  switch (a.LP) {
    case 768:
      if (out || da)
        return kind == 2 ? run_out<24, 32, 2>(a, st) : kind == 1 ? run_out<24, 32, 1>(a, st) : run_out2<24, 32, false>(a, st);
      return gather ? run_gather<24, 32, false>(a, st) : run_permg<24, 32>(a, st);
    case 255:
      if (out || da)
        return kind == 2 ? run_out<15, 17, 2>(a, st) : kind == 1 ? run_out<15, 17, 1>(a, st) : run_out<15, 17, 0>(a, st);
      return gather ? run_gather<15, 17, false>(a, st) : run_permg<15, 17>(a, st);
    case 50:
      if (out || da)
        return kind == 2 ? run_out<10, 5, 2>(a, st) : kind == 1 ? run_out<10, 5, 1>(a, st) : run_out<10, 5, 0>(a, st);
      return gather ? run_gather<10, 5, false>(a, st) : run_permg<10, 5>(a, st);
  }
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
