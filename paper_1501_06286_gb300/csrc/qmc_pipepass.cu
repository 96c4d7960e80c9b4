// qmc_pipepass.cu — persistent, double-buffered version of the
// register-resident pass kernel for the work-array passes (spectral pass B
// and inverse/un-permute pass C, forward and adjoint), pass lengths
// LP = P^2 with P = 16 or 32, panels of 8 complex columns.
//
// Each block loops over tiles (one line group of one panel: LP points x 8
// columns).  While it transforms tile i it has already issued the 16-byte
// cp.async copies of tile i+1 into the other shared buffer, so HBM reads
// stay in flight independently of how many blocks fit on an SM.  The
// shared buffer a tile lands in has the padded layout of the transposes and
// serves as their scratch, so a block needs two tile buffers and no more.
#include "qmc_pipe.cuh"

namespace qmc {

// ---------------------------------------------------------------------------
// First pass (scatter-add + forward transform), persistent and pipelined:
// tile = one first-pass line (n2) of one panel.  Its non-zero points come
// from the plan's padded gather table (at most kGatherMax entries per line,
// sorted by point), so the indices of a tile are loaded two tiles ahead with
// no dependent lookups, and the A row segments (64 bytes per entry) and the
// line's inter-pass twiddles w_L^{n2·k1} are fetched with cp.async one tile
// ahead.  Colliding entries (same point) are consecutive and summed in j
// order.
// ---------------------------------------------------------------------------
template <int P>
struct GatherSlot {
  static constexpr int LP = P * P;
  static constexpr int STG = kGatherMax * 8;             // staged A segments (complex)
  static constexpr int SLOT = STG + LP + kGatherMax / 2;  // + twiddles + point indices
};

template <int P>
__global__ void __launch_bounds__(P * 8, (P == 16 ? (QMC_TW_REGS ? 5 : 6) : 2))
    k_pipe_gather(const __grid_constant__ PassArgs a, int ntiles) {
  constexpr int LP = P * P;
  constexpr int SZ = (LP + P) * 8;
  constexpr int NT = P * 8;
  constexpr int STG = GatherSlot<P>::STG;
  constexpr int SLOT = GatherSlot<P>::SLOT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* S = tw + LP;
  cx<float>* slots = S + SZ;
  const int tid = threadIdx.x;
  const int w = tid & 7, t = tid >> 3;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += NT) tw[k] = twL[(int64_t)k * tstep];
  }
  MidTwiddles<P == 16 && QMC_TW_REGS, P> mtw{tw, t};
  __syncthreads();
  mtw.load();
  const int em = a.gp_em;
  const int nlg = a.n_linegroups;
  const int ge = tid >> 2, gq = tid & 3;  // prefetch role: entry, 16-byte quarter
  const float* Af = reinterpret_cast<const float*>(a.A);
  const int64_t pst = (int64_t)a.point_stride * 8;

  auto load_idx = [&](int tile, int& j, int& i) {
    i = -1;
    j = 0;
    if (tile < ntiles && ge < em) {
      const int ag = tile % nlg;
      j = a.gp_j[ag * em + ge];
      i = a.gp_i[ag * em + ge];
      if (i >= 0) {  // -1: padding
        i = chk(i, (int64_t)LP, a.err);
        j = chk(j, a.s_a, a.err);
      }
    }
  };
  auto prefetch = [&](int tile, cx<float>* slot, int j, int i) {
    const int ag = tile % nlg, p = tile / nlg;
    cx<float>* stg = slot;
    cx<float>* twl = slot + STG;
    int* idx = reinterpret_cast<int*>(twl + LP);
    if (ge < em) {
      if (gq == 0) idx[ge] = i;
      if (i >= 0) {
        const int col0 = 16 * p + 4 * gq;
        int bytes = (a.t - col0) * 4;
        bytes = bytes < 0 ? 0 : (bytes > 16 ? 16 : bytes);
        const float* src = bytes ? Af + (int64_t)j * a.lda + col0 : Af;
        cp_async16_zfill(stg + ge * 8 + 2 * gq, src, bytes);
      }
    }
    for (int k = tid; k < LP; k += NT) cp_async8(twl + k, twL + (int64_t)ag * k);
    cp_async_commit();
  };

  int tile = blockIdx.x;
  int jB, iB, jC, iC;
  load_idx(tile, jB, iB);
  if (tile < ntiles) prefetch(tile, slots, jB, iB);
  load_idx(tile + gridDim.x, jB, iB);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    cx<float>* cur = slots + (it & 1) * SLOT;
    cx<float>* nxt = slots + ((it + 1) & 1) * SLOT;
    const int next = tile + gridDim.x;
    load_idx(next + gridDim.x, jC, iC);
    if (next < ntiles) prefetch(next, nxt, jB, iB);
    else cp_async_commit();
    {  // zero the tile, 16 bytes per store (SZ is a multiple of 8 complex)
      float4* S4 = reinterpret_cast<float4*>(S);
#pragma unroll 4
      for (int e = tid; e < SZ / 2; e += NT) S4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    cp_async_wait<1>();
    __syncthreads();

    const int ag = tile % nlg, p = tile / nlg;
    const cx<float>* stg = cur;
    const cx<float>* twl = cur + STG;
    const int* idx = reinterpret_cast<const int*>(twl + LP);
    for (int pr = tid; pr < em * 8; pr += NT) {
      const int e = pr >> 3, w2 = pr & 7;
      const int i0 = idx[e];
      if (i0 >= 0 && (e == 0 || idx[e - 1] != i0)) {
        float re = 0.f, im = 0.f;
        for (int e2 = e; e2 < em && idx[e2] == i0; ++e2) {
          const cx<float> v = stg[e2 * 8 + w2];
          re += v.re;
          im += v.im;
        }
        const int c2 = 2 * ((p << 3) + w2);
        S[pidx<P>(i0, w2)] = mk<float>(c2 < a.t ? re * a.cscale[c2] : 0.f,
                                       c2 + 1 < a.t ? im * a.cscale[c2 + 1] : 0.f);
      }
    }
    __syncthreads();
    cx<float> x[P];
#pragma unroll
    for (int k = 0; k < P; ++k) x[k] = S[pidx<P>(t + P * k, w)];
    __syncthreads();
    pipe_fft<P, -1>(x, S, mtw, t, w);

    cx<float>* obase = reinterpret_cast<cx<float>*>(a.scratch) +
                       ((int64_t)p * a.L + (int64_t)ag * a.line_stride) * 8 + w;
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int i = t + P * k;
      obase[i * pst] = twmul<-1>(x[k], twl[i]);
    }
    jB = jC;
    iB = iC;
    __syncthreads();
  }
  cp_async_wait<0>();
}

template <int P>
static int run_pipe_gather(const PassArgs& a, cudaStream_t st) {
  constexpr int LP = P * P;
  const size_t smem =
      sizeof(cx<float>) * ((size_t)LP + (size_t)(LP + P) * 8 + 2 * (size_t)GatherSlot<P>::SLOT);
  static KernelSetup setup;
  int grid = 0;
  if (const int rc = setup_kernel(k_pipe_gather<P>, setup, smem, P * 8, &grid)) return rc;
  const int ntiles = a.n_linegroups * ((a.T + 7) >> 3);
  if (grid > ntiles) grid = ntiles;
  k_pipe_gather<P><<<grid, P * 8, smem, st>>>(a, ntiles);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

// The pipelined first pass: FP32 A with 16-byte aligned rows, 8-column
// panels, a padded gather table, pass length 256 or 1024.
int launch_pipe_gather(const PassArgs& a, cudaStream_t st) {
  if (a.gp_em < 1 || a.gp_em > kGatherMax || a.logW != 3 || a.a_f64 || a.split || !a.fwd || a.inv ||
      (a.lda % 4) != 0 || (((uintptr_t)a.A) & 15u) != 0 || a.twiddle >= 0)
    return QMC_ERR_UNSUPPORTED;
  if (a.LP == 256) return run_pipe_gather<16>(a, st);
  if (a.LP == 1024) return run_pipe_gather<32>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

template <int P, int MODE, int STORE, int SPEC>
static int run_pipe(const PassArgs& a, cudaStream_t st) {
  constexpr int LP = P * P;
  const size_t smem =
      sizeof(cx<float>) * ((size_t)LP + pipe_buffers<P>() * (size_t)PipeSlot<P, MODE, STORE>::SLOT);
  static KernelSetup setup;
  int grid = 0;
  if (const int rc = setup_kernel(k_pipe<P, MODE, STORE, SPEC>, setup, smem, P * 8, &grid)) return rc;
  const int ntiles = a.n_linegroups * ((a.T + 7) >> 3);
  if (grid > ntiles) grid = ntiles;
  k_pipe<P, MODE, STORE, SPEC><<<grid, P * 8, smem, st>>>(a, ntiles);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Plain un-permute pass (inverse P^2-point transform, FP32 store, no
// epilogues) over two panels per tile: 16 complex columns, so every output
// row of a tile receives one 128-byte run instead of two 64-byte runs from
// two tiles, which the scattered rows of B take at a much higher rate.
// Thread (t, w16): w16 < 16 the tile column, t < P the point group.
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ int pidx2(int i, int w) { return (i + i / P) * 16 + w; }

template <int P, int DIR, typename TW>
__device__ __forceinline__ void pipe_fft2(cx<float>* v, cx<float>* S, const TW& tw, int t, int w) {
  dftPp<P, DIR>(v);
#pragma unroll
  for (int k = 1; k < P; ++k) v[k] = twmul<DIR>(v[k], tw(k));
#pragma unroll
  for (int k = 0; k < P; ++k) S[pidx2<P>(k * P + t, w)] = v[k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < P; ++q) v[q] = S[pidx2<P>(t * P + q, w)];
  dftPp<P, DIR>(v);
  __syncthreads();
}

template <int P>
struct PipeOut2Shape {
  static constexpr int LP = P * P;
  static constexpr int NT = P * 16;
  static constexpr int SZ = (LP + P) * 16;
};

template <int P>
__global__ void __launch_bounds__(P * 16, 2) k_pipe_out2(const __grid_constant__ PassArgs a, int ntiles) {
  constexpr int LP = P * P, NT = P * 16, SZ = PipeOut2Shape<P>::SZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem_raw);
  cx<float>* bufs = tw + LP;
  const int tid = threadIdx.x;
  const int w = tid & 15, t = tid >> 4;
  const cx<float>* twL = reinterpret_cast<const cx<float>*>(a.twL);
  {
    const int tstep = a.L / LP;
    for (int k = tid; k < LP; k += NT) tw[k] = twL[(int64_t)k * tstep];
  }
  MidTwiddles<P == 16 && QMC_TW_REGS, P> mtw{tw, t};
  __syncthreads();
  mtw.load();
  const cx<float>* scratch_in = reinterpret_cast<const cx<float>*>(a.scratch);
  const int64_t pst = (int64_t)a.point_stride * 8;
  const int nlg = a.n_linegroups;
  const int npan = (a.T + 7) >> 3;

  auto prefetch = [&](int tile, cx<float>* dst) {
    const int ag = tile % nlg, pp = tile / nlg;
    const int64_t rb = (int64_t)ag * a.line_stride;
    const bool two = 2 * pp + 1 < npan;
#pragma unroll
    for (int q = 0; q < LP * 8 / NT; ++q) {
      const int c = tid + q * NT;  // 16-byte chunk: point c/8, columns 2*(c%8), +1 of the pair
      const int i = c >> 3, part = (c & 7) * 2;
      cx<float>* d = dst + pidx2<P>(i, part);
      if (part < 8 || two) {
        const int panel = 2 * pp + (part >> 3);
        cp_async16(d, scratch_in + ((int64_t)panel * a.L + rb) * 8 + i * pst + (part & 7));
      } else {
        d[0] = mk<float>(0.f, 0.f);
        d[1] = mk<float>(0.f, 0.f);
      }
    }
    cp_async_commit();
  };
  // output rows of a tile's points, loaded into registers one tile ahead
  auto load_rows = [&](int tile, int* rows) {
    const int ag = tile % nlg;
    const int* src = a.orow + (int64_t)ag * a.line_stride + (int64_t)t * a.point_stride;
    const int64_t step = (int64_t)P * a.point_stride;
#pragma unroll
    for (int k = 0; k < P; ++k) rows[k] = chk(__ldg(src + k * step), a.n_out, a.err);
  };
  int rows[P], rows_next[P];
  if ((int)blockIdx.x < ntiles) load_rows(blockIdx.x, rows);

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile, bufs);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    cx<float>* cur = bufs + (it & 1) * SZ;
    cx<float>* nxt = bufs + ((it + 1) & 1) * SZ;
    const int next = tile + gridDim.x;
    if (next < ntiles) {
      prefetch(next, nxt);
      load_rows(next, rows_next);
    } else {
      cp_async_commit();
    }
    cp_async_wait<1>();
    __syncthreads();
    cx<float> x[P];
#pragma unroll
    for (int k = 0; k < P; ++k) x[k] = cur[pidx2<P>(t + P * k, w)];
    __syncthreads();
    pipe_fft2<P, +1>(x, cur, mtw, t, w);

    const int c = ((tile / nlg) << 4) + w;
    if (c < a.T) {
      const int c2 = 2 * c;
      const bool pair = c2 + 1 < a.t;
      const float s0 = __ldg(a.cinv + c2), s1 = pair ? __ldg(a.cinv + c2 + 1) : 0.f;
      float* ocol = a.out + c2;
      if (pair && a.o_vec2) {
#pragma unroll
        for (int k = 0; k < P; ++k)
          *reinterpret_cast<float2*>(ocol + (int64_t)rows[k] * a.ldo) = make_float2(x[k].re * s0, x[k].im * s1);
      } else {
#pragma unroll
        for (int k = 0; k < P; ++k) {
          float* o = ocol + (int64_t)rows[k] * a.ldo;
          o[0] = x[k].re * s0;
          if (pair) o[1] = x[k].im * s1;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) rows[k] = rows_next[k];
  }
  cp_async_wait<0>();
}

template <int P>
static int run_pipe_out2(const PassArgs& a, cudaStream_t st) {
  constexpr int LP = P * P;
  const size_t smem = sizeof(cx<float>) * ((size_t)LP + 2 * (size_t)PipeOut2Shape<P>::SZ);
  static KernelSetup setup;
  int grid = 0;
  if (const int rc = setup_kernel(k_pipe_out2<P>, setup, smem, P * 16, &grid)) return rc;
  const int ntiles = a.n_linegroups * ((((a.T + 7) >> 3) + 1) >> 1);
  if (grid > ntiles) grid = ntiles;
  k_pipe_out2<P><<<grid, P * 16, smem, st>>>(a, ntiles);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int P>
static int run_pipe_p(const PassArgs& a, int store, cudaStream_t st) {
  const bool spectral = a.fwd && a.inv;
  const bool inv_only = !a.fwd && a.inv;
  if (spectral && store == ST_SCRATCH) {
    // the spectral pass of product_passes: contiguous points, store twiddle +1
    if (a.point_stride != 1 || a.twiddle != 1) return QMC_ERR_UNSUPPORTED;
    if (a.mul == 1) return run_pipe<P, PM_SPECTRAL, ST_SCRATCH, 1>(a, st);
    if (a.mul == 2) return run_pipe<P, PM_SPECTRAL, ST_SCRATCH, 2>(a, st);
    return QMC_ERR_UNSUPPORTED;
  }
  if (inv_only && a.twiddle == 0 && store == ST_OUT) {
    if (!a.split && !a.row_mean && !a.exp_sum && !a.col_off && !a.out_exp) {
      if constexpr (P == 16) return run_pipe_out2<P>(a, st);
      return run_pipe<P, PM_INV, ST_OUT, 1>(a, st);
    }
    return run_pipe<P, PM_INV, ST_OUT, 0>(a, st);
  }
  if (inv_only && a.twiddle == 0 && store == ST_DA) return run_pipe<P, PM_INV, ST_DA, 0>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

// Passes that read the work array (spectral pass or inverse/un-permute
// pass) with panels of 8 columns; anything else is QMC_ERR_UNSUPPORTED and
// the caller uses another kernel.
int launch_pipe_pass(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (load != LD_SCRATCH || a.logW != 3) return QMC_ERR_UNSUPPORTED;
  if (a.LP == 256) return run_pipe_p<16>(a, store, st);
  if (a.LP == 1024) return run_pipe_p<32>(a, store, st);
  return QMC_ERR_UNSUPPORTED;
}

// ---------------------------------------------------------------------------
// Sparse first pass (QMC_FIRST_PASS_SPARSE).  The first pass writes, for
// line k1 of the spectral pass and point n2,
//     Σ_{n1} a'[n1·L2 + n2]·w_L1^{-n1·k1}·w_L^{-n2·k1}
//   = Σ_{j: e_j ≡ n2 (mod L2)} a_j·w_L1^{-(n1_j·k1 mod L1)}·w_L^{-n2·k1},
// with e_j = n1_j·L2 + n2 and a' = P·A (Section 2.1's scatter-add).  When
// A has few rows per line the sum is cheaper than the length-L1 transform
// and its round trip through the work array, so the spectral pass forms
// its lines from the rows of A directly.
// ---------------------------------------------------------------------------
namespace {

// The packed rows of the sparse first pass (sparse_pack_row), one block row
// per entry.
__global__ void k_sparse_pack(const __grid_constant__ PassArgs a, int ncols) {
  sparse_pack_row(a, (int)blockIdx.x, ncols, (int)(blockIdx.y * blockDim.x + threadIdx.x),
                  (int)(gridDim.y * blockDim.x));
}

// Spectral pass of length LP = P^2 whose tiles are summed from the packed
// rows.  Thread (t, w) owns the points n2 ≡ t (mod P) of column w: it zeroes
// its slots of the shared tile, walks the entries of group t (the plan's
// entry list is grouped by n2 mod P) adding a_j·w_L1^{-(n1·k1 mod L1)}, and
// applies w_L^{-n2·k1} once per point when it reads its slots back.  No
// other thread touches those slots, so the sum needs no atomics; the
// entries of one point are added in j order.  The rest (forward transform,
// × H, inverse transform, store twiddle w_L^{+n2·k1}) is the spectral pass
// of k_pipe; H and the twiddles of the line are copied with cp.async while
// the sum runs.
template <int P>
__global__ void __launch_bounds__(P * 8, (pipe_min_blocks<P, PM_SPECTRAL, ST_SCRATCH, 1>()))
    k_pipe_sparse(const __grid_constant__ PassArgs a, int ntiles) {
  auto first_of = [&]() -> int { return (int)blockIdx.x; };
  auto step_of = [&]() -> int { return (int)gridDim.x; };
  auto sp_ld = [](const float2* q) -> float2 { return __ldg(q); };
#include "qmc_pipe_sparse_body.inc"
}

template <int P>
int run_pipe_sparse(const PassArgs& a, cudaStream_t st) {
  constexpr int LP = P * P;
  const size_t smem = sizeof(cx<float>) *
                      ((size_t)LP + (size_t)PipeSlot<P, PM_SPECTRAL, ST_SCRATCH>::SZ + 2 * (size_t)LP + a.n_linegroups);
  static KernelSetup setup;  // smem depends on L1: the occupancy is recomputed when it changes
  int grid = 0;
  if (const int rc = setup_kernel(k_pipe_sparse<P>, setup, smem, P * 8, &grid)) return rc;
  if (grid > ntiles_of(a)) grid = ntiles_of(a);
  k_pipe_sparse<P><<<grid, P * 8, smem, st>>>(a, ntiles_of(a));
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

}  // namespace

int launch_sparse_pack(const PassArgs& b, cudaStream_t st) {
  if (b.sp_s < 1 || !b.sp_ap || b.logW != 3) return QMC_ERR_UNSUPPORTED;
  const int ncols = ((b.T + 7) >> 3) * 8;
  const int nt = 256;
  int gy = (ncols + nt - 1) / nt;
  if (gy > 65535) gy = 65535;
  k_sparse_pack<<<dim3((unsigned)b.sp_s, (unsigned)gy), nt, 0, st>>>(b, ncols);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

// The spectral pass of product_passes (contiguous points, × H, store
// twiddle +1, 8-column panels) with its lines summed from the packed rows;
// pass length 256 or 1024, L1 <= 1024.
int launch_pipe_sparse(const PassArgs& b, cudaStream_t st) {
  if (b.logW != 3 || !(b.fwd && b.inv) || b.mul != 1 || b.twiddle != 1 || b.point_stride != 1 ||
      b.sp_s < 1 || !b.sp_ap || !b.sp_pos || !b.sp_gptr || b.n_linegroups > 1024 ||
      (int64_t)b.n_linegroups * b.LP != b.L)
    return QMC_ERR_UNSUPPORTED;
  if (b.LP == 256) return run_pipe_sparse<16>(b, st);
  if (b.LP == 1024) return run_pipe_sparse<32>(b, st);
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
