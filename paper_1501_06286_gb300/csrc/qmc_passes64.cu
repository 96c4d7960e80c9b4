// qmc_passes64.cu — FP64 instantiations of the pass kernel, used once per
// plan to transform the generator sequence z_k (Section 2.1) into its
// spectrum in double precision.
#include "qmc_pass_kernel.cuh"

namespace qmc {

template <int LOAD, int STORE>
static int run64(const PassArgs& a, cudaStream_t st) {
  const int items = a.LP << a.logM;
  int nt = (items + kEPT - 1) / kEPT;
  nt = ((nt + 31) / 32) * 32;
  if (nt < 32) nt = 32;
  if (nt > 512) return QMC_ERR_UNSUPPORTED;
  const bool rader = a.nst == 1 && (int)(a.rbits & 31u) == kRader257;
  const size_t smem = sizeof(cx<double>) * ((size_t)a.LP + 2 * (size_t)items +
                                            (rader ? 256 + 2 * ((size_t)1 << a.logM) : 0));
  // Opt in to the dynamic shared memory this launch needs (above the
  // 48 KB default); a refusal leaves no pending error behind.
  static KernelSetup setup;
  if (const int rc = setup_kernel(k_pass<double, LOAD, STORE>, setup, smem, nt, nullptr)) return rc;
  const int V = 1 << a.logV;
  dim3 grid((a.n_linegroups + V - 1) / V, (a.T + (1 << a.logW) - 1) >> a.logW);
  k_pass<double, LOAD, STORE><<<grid, nt, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

int launch_pass_f64(const PassArgs& a, int load, int store, cudaStream_t st) {
  if (load == LD_DENSE64 && store == ST_SCRATCH) return run64<LD_DENSE64, ST_SCRATCH>(a, st);
  if (load == LD_SCRATCH && store == ST_SCRATCH) return run64<LD_SCRATCH, ST_SCRATCH>(a, st);
  return QMC_ERR_UNSUPPORTED;
}

}  // namespace qmc
