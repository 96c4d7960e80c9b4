// qmc_fastpass.cu — launches of the register-resident pass kernel k_fast
// for the square pass lengths LP = P^2 (P = 16: 256 points, P = 32: 1024
// points): one tile of 8 lines per block, the tile of qmc_fast.cuh.

#include "qmc_fast.cuh"

namespace qmc {

template <int P, int LOAD, int STORE, int MODE>
__global__ void __launch_bounds__(P * kFastM, (P == 16 ? 6 : 2))
    k_fast(const __grid_constant__ PassArgs a) {
  constexpr int M = kFastM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned bx = blockIdx.x, by = blockIdx.y;
#include "qmc_fast_body.inc"
}

template <int P, int LOAD, int STORE, int MODE>
static int run_fast(const PassArgs& a, cudaStream_t st) {
  constexpr int LP = P * P;
  const size_t smem = sizeof(cx<float>) * ((size_t)LP + (size_t)(LP + P) * kFastM);
  static KernelSetup setup;
  if (const int rc = setup_kernel(k_fast<P, LOAD, STORE, MODE>, setup, smem, P * kFastM, nullptr)) return rc;
  const int V = kFastM >> a.logW;
  dim3 grid((a.n_linegroups + V - 1) / V, (a.T + (1 << a.logW) - 1) >> a.logW);
  k_fast<P, LOAD, STORE, MODE><<<grid, P * kFastM, smem, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

template <int P>
static int dispatch_fast(const PassArgs& a, int load, int store, int mode, cudaStream_t st) {
  if (mode == FM_FWD && load == LD_GATHER_A && store == ST_SCRATCH)
    return run_fast<P, LD_GATHER_A, ST_SCRATCH, FM_FWD>(a, st);
  if (mode == FM_FWD && load == LD_PERM_G && store == ST_SCRATCH)
    return run_fast<P, LD_PERM_G, ST_SCRATCH, FM_FWD>(a, st);
  if (mode == FM_SPECTRAL && load == LD_SCRATCH && store == ST_SCRATCH)
    return run_fast<P, LD_SCRATCH, ST_SCRATCH, FM_SPECTRAL>(a, st);
  if (mode == FM_SPECTRAL && load == LD_GATHER_A && store == ST_OUT)
    return run_fast<P, LD_GATHER_A, ST_OUT, FM_SPECTRAL>(a, st);
  if (mode == FM_SPECTRAL && load == LD_PERM_G && store == ST_DA)
    return run_fast<P, LD_PERM_G, ST_DA, FM_SPECTRAL>(a, st);
  if (mode == FM_INV && load == LD_SCRATCH && store == ST_OUT)
    return run_fast<P, LD_SCRATCH, ST_OUT, FM_INV>(a, st);
  if (mode == FM_INV && load == LD_SCRATCH && store == ST_DA)
    return run_fast<P, LD_SCRATCH, ST_DA, FM_INV>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

bool fast_pass_supported(int LP) { return LP == 256 || LP == 1024; }

// Runs pass `a` with the register-resident kernel.  The pass is given by
// its flags: forward only (pass A), forward + spectrum + inverse (pass B,
// or a single pass), inverse only (pass C).  The tile is 8 lines: one
// panel of W <= 8 complex columns times 8/W line groups.
int launch_fast_pass(PassArgs a, int load, int store, cudaStream_t st) {
  int mode;
  if (a.fwd && a.inv) mode = FM_SPECTRAL;
  else if (a.fwd) mode = FM_FWD;
  else mode = FM_INV;
  if (a.logW > 3) return QMC_ERR_UNSUPPORTED;
  a.logV = 3 - a.logW;
  a.logM = 3;
  if (a.LP == 256) return dispatch_fast<16>(a, load, store, mode, st);
  if (a.LP == 1024) return dispatch_fast<32>(a, load, store, mode, st);
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
