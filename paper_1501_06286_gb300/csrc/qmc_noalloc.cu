// qmc_noalloc.cu — qmc_matmul_noalloc: the forward product with its scratch
// (column statistics and the L x T work array between the FFT passes) in a
// fixed device array of this library instead of plan-owned memory, so that
// the call itself allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it until the process exits.  Host code cannot use the
// variable's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current)
// and keeps it for the life of the process.  That address belongs to the
// device's current context: after cudaDeviceReset (or anything else that
// destroys the primary context) the kept address is stale, so a caller that
// resets a device must not call this entry point on it again in the same
// process.  Every call shares the one array: calls whose kernels overlap on
// the GPU (two streams, two host threads) race on it.  Nothing
// in it needs to start at zero: every pass writes the elements the next
// pass reads.
#include <mutex>

#include "qmc_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

void* g_static_addr[qmc::kMaxDevices] = {};
std::mutex g_static_mutex;

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

using namespace qmc;

extern "C" int qmc_matmul_noalloc(void* plan, const void* A, int64_t lda, int32_t t, int32_t a_dtype,
                                  float* out, int64_t ldo, void* stream) {
  if (!plan || !A || !out) return QMC_ERR_INVALID;
  Plan& p = *static_cast<Plan*>(plan);
  if (p.pset) return QMC_ERR_UNSUPPORTED;  // Korobov p-set plans: qmc_matmul only
  if (t < 1 || lda < t || ldo < t) return QMC_ERR_SHAPE;
  if (a_dtype != QMC_DTYPE_F32 && a_dtype != QMC_DTYPE_F64) return QMC_ERR_INVALID;
  if (p.prec == QMC_PREC_FP32_SPLIT && a_dtype != QMC_DTYPE_F64) return QMC_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;

  // Size check before any device work: statistics, then the work array.
  const int T = p.prec == QMC_PREC_FP32_SPLIT ? t : (t + 1) / 2;
  int W = 1;
  while (W < 8 && W < T) W <<= 1;
  const size_t stats = round256(colstats_bytes(p.s, t));
  const size_t work = p.L2 == 1 ? 0
                                : (size_t)((T + W - 1) / W) * (size_t)p.L * (size_t)W * sizeof(cx<float>);
  if (stats + work > kStaticScratchBytes) return QMC_ERR_SCRATCH;

  // Device address of the static array, looked up once per device.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return QMC_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return QMC_ERR_CUDA;
      }
      g_static_addr[dev] = ptr;
    }
    base = g_static_addr[dev];
  }
  unsigned char* stats_ptr = static_cast<unsigned char*>(base);
  unsigned char* work_ptr = stats_ptr + stats;

  float *cscale = nullptr, *cinv = nullptr;
  int rc = launch_colstats(stats_ptr, A, lda, p.s, t, a_dtype == QMC_DTYPE_F64, 0, 1.f, p.phi0,
                           p.has_row0 ? out : nullptr, nullptr, nullptr, &cscale, &cinv, st, p.d_err);
  if (rc) return rc;

  PassArgs base_args{};
  base_args.T = T;
  base_args.t = t;
  base_args.A = A; base_args.lda = lda; base_args.a_f64 = a_dtype == QMC_DTYPE_F64;
  base_args.split = p.prec == QMC_PREC_FP32_SPLIT;
  base_args.a_vec2 = !base_args.a_f64 && (lda % 2 == 0) && (((uintptr_t)A & 7u) == 0);
  base_args.out = out; base_args.ldo = ldo;
  base_args.o_vec2 = (ldo % 2 == 0) && (((uintptr_t)out & 7u) == 0);
  base_args.inv_t = 1.0f / (float)t;
  base_args.cscale = cscale;
  base_args.cinv = cinv;
  base_args.scratch = work_ptr;
  base_args.twL = p.d_tw;
  base_args.H = p.d_H;
  base_args.row_ptr = p.d_row_ptr;
  base_args.jlist = p.d_jlist;
  base_args.bucket_ptr = p.d_bucket_ptr;
  base_args.blist = p.d_blist;
  base_args.orow = p.d_orow;
  base_args.err = p.d_err;
  base_args.n_out = p.out_rows;
  base_args.s_a = p.s;
  base_args.L = (int)p.L;
  base_args.rader = p.d_rader32;
  base_args.rader_perm = p.d_rader_perm;

  auto run = [&](const PassArgs& a, int load, int store) {
    if (p.pass_kernel != QMC_KERNEL_GENERIC && fast_pass_supported(a.LP)) {
      const int r = launch_fast_pass(a, load, store, st);
      if (r != QMC_ERR_UNSUPPORTED) return r;
    }
    return launch_pass(a, 0, load, store, st);
  };

  if (p.L2 == 1) {
    PassArgs a = base_args;
    a.LP = p.L1; a.nst = p.rad1.n; a.rbits = p.rad1.packed();
    a.point_stride = 1; a.line_stride = 1; a.n_linegroups = 1;
    a.fwd = 1; a.inv = 1; a.mul = 1; a.twiddle = 0;
    if (choose_tile(a.LP, T, 8, 1, &a.logW, &a.logV)) return QMC_ERR_UNSUPPORTED;
    a.logV = 0;
    a.logM = a.logW;
    return run(a, LD_GATHER_A, ST_OUT);
  }
  PassArgs a = base_args;
  a.LP = p.L1; a.nst = p.rad1.n; a.rbits = p.rad1.packed();
  a.point_stride = p.L2; a.line_stride = 1; a.n_linegroups = p.L2;
  a.fwd = 1; a.twiddle = -1;
  if (choose_tile(a.LP, T, 8, a.n_linegroups, &a.logW, &a.logV)) return QMC_ERR_UNSUPPORTED;
  a.logM = a.logW + a.logV;
  if ((rc = run(a, LD_GATHER_A, ST_SCRATCH))) return rc;

  PassArgs b = base_args;
  b.LP = p.L2; b.nst = p.rad2.n; b.rbits = p.rad2.packed();
  b.point_stride = 1; b.line_stride = p.L2; b.n_linegroups = p.L1;
  b.fwd = 1; b.inv = 1; b.mul = 1; b.twiddle = +1;
  if (choose_tile(b.LP, T, 8, b.n_linegroups, &b.logW, &b.logV)) return QMC_ERR_UNSUPPORTED;
  b.logM = b.logW + b.logV;
  if ((rc = run(b, LD_SCRATCH, ST_SCRATCH))) return rc;

  PassArgs c = base_args;
  c.LP = p.L1; c.nst = p.rad1.n; c.rbits = p.rad1.packed();
  c.point_stride = p.L2; c.line_stride = 1; c.n_linegroups = p.L2;
  c.inv = 1;
  if (choose_tile(c.LP, T, 8, c.n_linegroups, &c.logW, &c.logV)) return QMC_ERR_UNSUPPORTED;
  c.logM = c.logW + c.logV;
  return run(c, LD_SCRATCH, ST_OUT);
}
