// qmc_batch.cu — products over many plans (uneven N, s, t) in one call.
//
// Two ways to run a batch:
//
// GRAPH (default).  The first call captures every problem's product (column
// statistics and FFT passes, each with its fastest kernel) into one CUDA
// graph whose branches run problems concurrently, after the autotuner has
// picked, per problem, the transform's factorisation, the pass kernel and
// the first-pass mode (cached per problem shape) and, for the batch, the
// number of branches.  Later calls with the same pointers replay the graph: one
// launch per call.
//
// PERSISTENT.  After the column statistics of every problem (two
// launches for the whole batch), one kernel launch drains a work queue of
// (problem, stage, chunk of tiles) items in stage-major order: every
// first-stage chunk of every problem, then every second-stage chunk, then
// the third stage (a stage is a pass, or the row packing of the sparse
// first pass).  A chunk of stage k waits until all chunks of stage k-1 of
// its problem are done (per-(problem, stage) completion counters).  Chunks are claimed in queue order by resident
// blocks, so every chunk a claimed chunk waits for was claimed earlier by
// a running block: the waits always end.  Each wait is still bounded: past
// the limit the block latches QMC_ERR_TIMEOUT in the batch's error word,
// raises the abort flag every block polls, and returns.
//
// A queue item runs the tile loop of the pass's specialised persistent
// kernel where the pass has one in the queue's 256-thread shape — the
// 768-point first pass (term-by-term lines and lines from the padded
// gather table), the 1024-point spectral pass, plain or summed from the
// packed rows of the sparse first pass (with the packing as the problem's
// first stage), and the 768-point plain un-permute pass, i.e. every pass
// of the 768 x 1024 transform — on a chunk of tiles, and the
// generic shared-memory tile otherwise.  A block claims its next chunk
// while it works on the current one, and it checks a chunk's dependency
// and loads its arguments only when the chunk belongs to another item than
// its previous one.  A claimed chunk waits only for chunks earlier in the
// queue, so the lowest unfinished chunk is always running and the launch
// always progresses.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "qmc_fast.cuh"
#include "qmc_pass_kernel.cuh"
#include "qmc_pipe.cuh"
#include "qmc_pqpipe.cuh"

namespace qmc {

// What a queue item runs.
enum QueueKind : int {
  QK_GENERIC = 0,    // pass_tile, any pass (load/store modes in the item)
  QK_DIRECT768 = 1,  // 768-point first pass, term-by-term lines (a pair counts as two lines)
  QK_GATHER768 = 2,  // 768-point first pass, lines from the padded gather table
  QK_SPEC1024 = 3,   // 1024-point spectral pass (× H)
  QK_OUT768 = 4,     // 768-point un-permute pass, plain FP32 store
  QK_PACK = 5,       // sparse first pass: packed rows of A (one tile per entry)
  QK_SPARSE1024 = 6, // 1024-point spectral pass summed from the packed rows
  QK_FAST256 = 7,    // any pass of length 256: register tile of 16 lines (load/store modes in the item)
};

constexpr int kQueueThreads = 256;

struct BatchItem {
  PassArgs a;
  int kind;
  int load, store;  // QK_GENERIC: load / store modes
  int gx;           // QK_GENERIC: tiles along the line groups
  int teams;        // QK_GENERIC: tiles in flight per block (2: one per half-block)
  int sbytes;       // QK_GENERIC: shared memory of one tile
  int ntiles;       // tiles of the item
  int chunk;        // tiles per claim
  int first;        // queue index of the item's first chunk
  int nchunks;      // chunks of the item: chunk c takes tiles c, c + nchunks, ...
  int group;        // (problem, pass) counter this item's chunks complete
  int dep;          // counter it waits for, -1 for none
  int need;         // completed chunks that counter must reach
};

namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The specialised tile loops on tiles [first, ntiles) with step 1: the same
// text as the stand-alone persistent kernels, `a` the item's arguments.
template <int LP, bool SPLIT>
__device__ __forceinline__ void q_direct(const PassArgs& a, int q_first, int q_step, int ntiles) {
  auto first_of = [&]() -> int { return q_first; };
  auto step_of = [&]() -> int { return q_step; };
  // virtual lines: the pairs' lines 2λ, 2λ+1 first, then the single lines
  auto direct_lines = [&]() -> int { return 2 * a.n_pair + a.n_direct; };
  auto direct_line = [&](int v) -> int {
    const int np2 = 2 * a.n_pair;
    return v < np2 ? __ldg(a.lines + (v >> 1)) + (v & 1) : __ldg(a.lines + a.n_pair + (v - np2));
  };
#include "qmc_pq_direct_body.inc"
}

template <int P, int Q, bool SPLIT>
__device__ __forceinline__ void q_gather(const PassArgs& a, int q_first, int q_step, int ntiles) {
  auto first_of = [&]() -> int { return q_first; };
  auto step_of = [&]() -> int { return q_step; };
#include "qmc_pqpipe_gather_body.inc"
}

template <int P, int Q, int KIND>
__device__ __forceinline__ void q_out(const PassArgs& a, int q_first, int q_step, int ntiles) {
  auto first_of = [&]() -> int { return q_first; };
  auto step_of = [&]() -> int { return q_step; };
#include "qmc_pqpipe_out_body.inc"
}

template <int P, int MODE, int STORE, int SPEC>
__device__ __forceinline__ void q_pipe(const PassArgs& a, int q_first, int q_step, int ntiles) {
  auto first_of = [&]() -> int { return q_first; };
  auto step_of = [&]() -> int { return q_step; };
#include "qmc_pipe_body.inc"
}

template <int P>
__device__ __forceinline__ void q_sparse(const PassArgs& a, int q_first, int q_step, int ntiles) {
  auto first_of = [&]() -> int { return q_first; };
  auto step_of = [&]() -> int { return q_step; };
  // the packed rows were written earlier in this launch: plain (coherent)
  // loads, not the read-only path; they stay in L1 for the tiles that
  // follow, like the stand-alone kernel's
  auto sp_ld = [](const float2* q) -> float2 { return *q; };
#include "qmc_pipe_sparse_body.inc"
}

// Register tiles of length 256 (16 lines, 256 threads): tiles first,
// first + step, ... below n of a tile grid gx wide.
template <int LOAD, int STORE, int MODE>
__device__ __forceinline__ void q_fast_tiles(const PassArgs& a, int gx, int first, int step, int n) {
  constexpr int P = 16, M = 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int tile = first; tile < n; tile += step) {
    const unsigned bx = (unsigned)(tile % gx), by = (unsigned)(tile / gx);
    {
#include "qmc_fast_body.inc"
    }
    __syncthreads();  // the next tile rewrites the shared tile
  }
}

__device__ __noinline__ void q_fast(const PassArgs& a, int load, int store, int gx, int first, int step, int n) {
  if (load == LD_GATHER_A && store == ST_SCRATCH) q_fast_tiles<LD_GATHER_A, ST_SCRATCH, FM_FWD>(a, gx, first, step, n);
  else if (load == LD_SCRATCH && store == ST_SCRATCH) q_fast_tiles<LD_SCRATCH, ST_SCRATCH, FM_SPECTRAL>(a, gx, first, step, n);
  else if (load == LD_SCRATCH && store == ST_OUT) q_fast_tiles<LD_SCRATCH, ST_OUT, FM_INV>(a, gx, first, step, n);
  else if (load == LD_GATHER_A && store == ST_OUT) q_fast_tiles<LD_GATHER_A, ST_OUT, FM_SPECTRAL>(a, gx, first, step, n);
}

__device__ __forceinline__ void q_pack(const PassArgs& a, int first, int step, int n) {
  const int ncols = ((a.T + 7) >> 3) * 8;
  for (int q = first; q < n; q += step) sparse_pack_row(a, q, ncols, (int)threadIdx.x, (int)blockDim.x);
}

static_assert(PqPipeShape<24, 32>::NT == kQueueThreads && PqDirectShape<768>::NT == kQueueThreads &&
                  32 * 8 == kQueueThreads && 16 * 16 == kQueueThreads,
              "the specialised tile loops of the queue run on 256 threads");

// Half of the queue's block (128 threads) with named barrier 1 + half.
struct HalfTeam {
  static constexpr bool kWhole = false;
  int half;
  __device__ __forceinline__ int tid() const { return (int)threadIdx.x & 127; }
  __device__ __forceinline__ int nt() const { return 128; }
  __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, 128;" ::"r"(1 + half) : "memory"); }
};

template <typename TM>
__device__ __forceinline__ void generic_tile(const PassArgs& a, int load, int store, int bx, int by,
                                             unsigned char* smem, const TM& tm) {
  if (load == LD_GATHER_A && store == ST_SCRATCH) pass_tile<float, LD_GATHER_A, ST_SCRATCH>(a, bx, by, smem, tm);
  else if (load == LD_SCRATCH && store == ST_SCRATCH) pass_tile<float, LD_SCRATCH, ST_SCRATCH>(a, bx, by, smem, tm);
  else if (load == LD_SCRATCH && store == ST_OUT) pass_tile<float, LD_SCRATCH, ST_OUT>(a, bx, by, smem, tm);
  else if (load == LD_GATHER_A && store == ST_OUT) pass_tile<float, LD_GATHER_A, ST_OUT>(a, bx, by, smem, tm);
  tm.sync();  // the team's next tile reuses its shared buffers
}

// Generic tiles first, first + step, ... below n: with two teams, half h
// of the block takes every other one of them (h first) in its own part of
// the shared memory, so that two tiles' memory latencies overlap in one
// block.
__device__ __noinline__ void q_generic(const PassArgs& a, int load, int store, int gx, int teams, int sbytes,
                                       int first, int step, int n, unsigned char* smem) {
  if (teams == 2) {
    const HalfTeam tm{(int)threadIdx.x >> 7};
    for (int tile = first + tm.half * step; tile < n; tile += 2 * step)
      generic_tile(a, load, store, tile % gx, tile / gx, smem + (size_t)tm.half * sbytes, tm);
  } else {
    for (int tile = first; tile < n; tile += step)
      generic_tile(a, load, store, tile % gx, tile / gx, smem, BlockTeam());
  }
}

// The loop keeps its state in shared memory (and the kernel parameters),
// so that nothing of it stays live in registers across a tile loop: each
// loop has the registers its stand-alone kernel has.
__global__ void __launch_bounds__(kQueueThreads, 2)
    k_batch(const BatchItem* __restrict__ items, const int* __restrict__ chunk_item, int total_chunks,
            int* counters, int* queue, int* err, long long wait_cycles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PassArgs s_a;
  __shared__ int s_chunk, s_item, s_abort, s_cur, s_next;  // s_next: the chunk claimed ahead
  constexpr int kWords = (int)(sizeof(PassArgs) / sizeof(int));
  static_assert(sizeof(PassArgs) % sizeof(int) == 0, "PassArgs copied as words");
  if (threadIdx.x == 0) {
    s_next = atomicAdd(queue, 1);
    s_cur = -1;  // item whose arguments s_a holds, its dependency met
  }
  for (;;) {
    __syncthreads();  // the previous chunk is done with the shared buffers
    if (threadIdx.x == 0) {
      const int c = ld_acquire(err) != 0 ? total_chunks : s_next;
      s_chunk = c;
      if (c < total_chunks) {
        s_item = __ldg(chunk_item + c);
        s_next = atomicAdd(queue, 1);
      }
      s_abort = 0;
    }
    __syncthreads();
    if (s_chunk >= total_chunks) return;
    if (s_item != s_cur) {
      const BatchItem* it = items + s_item;
      const int dep = it->dep;
      if (threadIdx.x == 0 && dep >= 0) {
        const int need = it->need;
        const long long t0 = clock64();
        while (ld_acquire(counters + dep) < need) {
          if (ld_acquire(err) != 0) { s_abort = 1; break; }
          if (clock64() - t0 > wait_cycles) {
            atomicOr(err, kErrTimeout);
            s_abort = 1;
            break;
          }
          __nanosleep(256);
        }
        __threadfence();
      }
      const int* src = reinterpret_cast<const int*>(&it->a);
      int* dst = reinterpret_cast<int*>(&s_a);
      for (int q = threadIdx.x; q < kWords; q += blockDim.x) dst[q] = src[q];
      __syncthreads();
      if (s_abort) return;
      if (threadIdx.x == 0) s_cur = s_item;
    }
    {
      const BatchItem* it = items + s_item;
      // chunk c of an item takes its tiles c, c + nchunks, ...: the chunks
      // that run at the same time cover neighbouring tiles, as the blocks of
      // a stand-alone persistent kernel do
      const int c = s_chunk - it->first, step = it->nchunks, n = it->ntiles;
      switch (it->kind) {
        case QK_DIRECT768: q_direct<768, false>(s_a, c, step, n); break;
        case QK_GATHER768: q_gather<24, 32, false>(s_a, c, step, n); break;
        case QK_SPEC1024: q_pipe<32, PM_SPECTRAL, ST_SCRATCH, 1>(s_a, c, step, n); break;
        case QK_OUT768: q_out<24, 32, 0>(s_a, c, step, n); break;
        case QK_PACK: q_pack(s_a, c, step, n); break;
        case QK_SPARSE1024: q_sparse<32>(s_a, c, step, n); break;
        case QK_FAST256: q_fast(s_a, it->load, it->store, it->gx, c, step, n); break;
        default: q_generic(s_a, it->load, it->store, it->gx, it->teams, it->sbytes, c, step, n, smem_raw); break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(counters + items[s_item].group, 1);
    }
  }
}

size_t generic_tile_smem(const PassArgs& a) {
  const bool rader = a.nst == 1 && (int)(a.rbits & 31u) == kRader257;
  const size_t items = (size_t)a.LP << a.logM;
  return sizeof(cx<float>) * ((size_t)a.LP + 2 * items + (rader ? 256 + 2 * ((size_t)1 << a.logM) : 0));
}

// Dynamic shared memory of each specialised tile loop (the layouts of the
// stand-alone launches).
constexpr size_t kSmemDirect768 = sizeof(cx<float>) * (768 + 2 * (size_t)PqDirectShape<768>::SLOT);
constexpr size_t kSmemGather768 =
    sizeof(cx<float>) * (768 + (size_t)PqPipeShape<24, 32>::SZ + 2 * (size_t)PqPipeShape<24, 32>::GATHER_SLOT);
constexpr size_t kSmemSpec1024 =
    sizeof(cx<float>) * (1024 + pipe_buffers<32>() * (size_t)PipeSlot<32, PM_SPECTRAL, ST_SCRATCH>::SLOT);
constexpr size_t kSmemOut768 = sizeof(cx<float>) * (768 + 2 * (size_t)PqPipeShape<24, 32>::OUT_SLOT);
size_t smem_sparse1024(int L1) {
  return sizeof(cx<float>) * (1024 + (size_t)PipeSlot<32, PM_SPECTRAL, ST_SCRATCH>::SZ + 2 * 1024 + (size_t)L1);
}
// generic tiles are narrowed (fewer line groups per tile) to fit in this
// much, so that two blocks stay resident per SM
constexpr size_t kQueueSmemCap = kSmemOut768;

}  // namespace
}  // namespace qmc

using namespace qmc;

namespace {

struct Batch {
  std::vector<Plan*> plans;
  std::vector<int32_t> t;
  int mode = QMC_BATCH_GRAPH;
  int branches = 0;              // 0: autotune
  long long wait_us = 1000000;   // bounded wait of the persistent mode
  int test_block_item = -1;      // test hook: this item's dependency never completes
  // graph mode
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> br;
  std::vector<cudaEvent_t> ev;
  cudaGraphExec_t exec = nullptr;
  unsigned long long graph_kernels = 0;  // kernel launches captured in `exec`
  std::vector<const void*> keyA;
  std::vector<float*> keyOut;
  std::vector<int64_t> keyLda, keyLdo;
  bool tuned = false;
  // persistent mode
  // the queue's description — items, column-statistics jobs, the item of
  // each chunk — as one blob, uploaded through pinned memory only when it
  // differs from the previous call's
  unsigned char* d_blob = nullptr;
  unsigned char* h_stage = nullptr;  // pinned
  size_t cap_blob = 0;
  std::vector<unsigned char> last_blob;
  cudaEvent_t up_ev = nullptr;       // the last upload from h_stage
  cudaEvent_t done_ev = nullptr;     // the last queue launch (a later call on another stream waits for it)
  int* d_counters = nullptr;  // [3 per problem] + queue head
  int* d_err = nullptr;
  int cap_counters = 0;
  std::vector<BatchItem> h_items;
  std::vector<int> h_chunk_item;
};

void free_graph(Batch& b) {
  if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
}

int capture(Batch& b, const float* const* A, const int64_t* lda, float* const* out,
            const int64_t* ldo, int nbranch) {
  if ((int)b.br.size() < nbranch) return QMC_ERR_INVALID;
  if (cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return QMC_ERR_CUDA;
  }
  int rc = QMC_OK;
  cudaEventRecord(b.ev[0], b.cap);
  for (int k = 0; k < nbranch; ++k) cudaStreamWaitEvent(b.br[k], b.ev[0], 0);
  const unsigned long long launches0 = launch_total();
  // largest problems first so that branches start with the long work
  std::vector<int> order(b.plans.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    return (double)b.plans[x]->L * b.t[x] > (double)b.plans[y]->L * b.t[y];
  });
  for (size_t q = 0; q < order.size() && rc == QMC_OK; ++q) {
    const int i = order[q];
    rc = qmc_matmul(b.plans[i], A[i], lda[i], b.t[i], QMC_DTYPE_F32, out[i], ldo[i], nullptr, nullptr,
                    b.br[q % nbranch]);
  }
  for (int k = 0; k < nbranch; ++k) {
    cudaEventRecord(b.ev[1 + k], b.br[k]);
    cudaStreamWaitEvent(b.cap, b.ev[1 + k], 0);
  }
  // captured launches ran nothing yet: take them back out of the count and
  // add them at every replay instead
  const unsigned long long captured = launch_total() - launches0;
  add_launches(-(long long)captured);
  b.graph_kernels = captured;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(b.cap, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return rc ? rc : QMC_ERR_CUDA;
  }
  if (rc) { cudaGraphDestroy(g); return rc; }
  free_graph(b);
  if (cudaGraphInstantiate(&b.exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return QMC_ERR_CUDA;
  }
  cudaGraphDestroy(g);
  b.keyA.assign(A, A + b.plans.size());
  b.keyOut.assign(out, out + b.plans.size());
  b.keyLda.assign(lda, lda + b.plans.size());
  b.keyLdo.assign(ldo, ldo + b.plans.size());
  return QMC_OK;
}

int launch_graph(Batch& b, cudaStream_t st) {
  if (cudaGraphLaunch(b.exec, st) != cudaSuccess) {
    cudaGetLastError();
    return QMC_ERR_CUDA;
  }
  add_launches((long long)b.graph_kernels);
  return QMC_OK;
}

float time_ms(cudaStream_t st, const std::function<int()>& f, int reps, int* rc) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  *rc = f();  // warm-up
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps && !*rc; ++r) *rc = f();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return reps ? ms / reps : ms;
}

// ---------------------------------------------------------------------------
// Autotuner.  Per problem it times every candidate configuration — the
// transform's factorisation L = L1·L2 (the default and the next splits with
// both factors at most 1024, shortest longer factor first), the pass kernel
// (fastest available, or the generic shared-memory kernel) and, where the
// plan offers it, the first-pass mode (transform or sparse) — and keeps the
// fastest; then it picks the number of graph branches for the batch.
// Choices are cached for the process under (kind, L, ⌊log2 s⌋, ⌊log2 t⌋,
// compute capability), so problems of the same shape are timed once; with
// QMC_AUTOTUNE_CACHE naming a file, the cache is read from it on first use
// and every new choice is appended as one text line
//   kind L log2s log2t arch L1 kernel first ms
// ---------------------------------------------------------------------------
struct TuneKey {
  int kind;
  int64_t L;
  int sb, tb, arch;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, L, sb, tb, arch) < std::tie(o.kind, o.L, o.sb, o.tb, o.arch);
  }
};
struct TuneChoice {
  int L1, kernel, first;
  float ms;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;
bool g_tune_loaded = false;

int floor_log2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= v) ++l;
  return l;
}

void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("QMC_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  TuneKey k{};
  TuneChoice c{};
  long long L = 0;
  while (fscanf(f, "%d %lld %d %d %d %d %d %d %f", &k.kind, &L, &k.sb, &k.tb, &k.arch, &c.L1, &c.kernel,
                &c.first, &c.ms) == 9) {
    k.L = L;
    g_tune[k] = c;
  }
  fclose(f);
}

void tune_cache_append(const TuneKey& k, const TuneChoice& c) {
  const char* path = getenv("QMC_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%d %lld %d %d %d %d %d %d %.5f\n", k.kind, (long long)k.L, k.sb, k.tb, k.arch, c.L1, c.kernel,
          c.first, c.ms);
  fclose(f);
}

// Candidate first factors L1 of L: the current (default) one first, then
// (for two-pass plans) up to `extra` other splits a·b = L, a <= b <= 1024,
// both of supported radices, by increasing b.
std::vector<int> split_candidates(const Plan& p, int extra) {
  std::vector<int> out{p.L1};
  if (p.L2 == 1) return out;  // one pass: every split would add a pass
  std::vector<std::pair<int64_t, int>> alt;
  for (int64_t a = 2; a <= 1024 && a * a <= p.L; ++a) {
    if (p.L % a) continue;
    const int64_t b = p.L / a;
    if (b > 1024 || a == p.L1) continue;
    Radices ra, rb;
    if (!factor_radices((int)a, &ra) || !factor_radices((int)b, &rb)) continue;
    alt.push_back({b, (int)a});
  }
  std::sort(alt.begin(), alt.end());
  for (size_t k = 0; k < alt.size() && (int)k < extra; ++k) out.push_back(alt[k].second);
  return out;
}

int apply_choice(Plan& p, const TuneChoice& c, int t) {
  int rc = qmc_plan_set_option(&p, QMC_OPT_FFT_SPLIT, c.L1 == (int)p.L ? p.L : c.L1);
  if (rc) return rc;
  p.pass_kernel = c.kernel;
  p.first_pass = c.first;
  return qmc_plan_reserve(&p, t);  // the capture that follows must not allocate
}

int tune_problem(Plan& p, int t, const float* A, int64_t lda, float* out, int64_t ldo, int arch,
                 cudaStream_t st) {
  const TuneKey key{p.kind, p.L, floor_log2(p.s), floor_log2(t), arch};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    const auto it = g_tune.find(key);
    if (it != g_tune.end()) return apply_choice(p, it->second, t);
  }
  TuneChoice best{p.L1, p.pass_kernel, p.first_pass, 1e30f};
  int rc = QMC_OK;
  for (int L1 : split_candidates(p, 3)) {
    if ((rc = qmc_plan_set_option(&p, QMC_OPT_FFT_SPLIT, L1))) return rc;
    if ((rc = qmc_plan_reserve(&p, t))) return rc;
    const bool sparse_ok = p.sp_P != 0;
    for (int k : {QMC_KERNEL_AUTO, QMC_KERNEL_GENERIC}) {
      for (int fp : {QMC_FIRST_PASS_TRANSFORM, QMC_FIRST_PASS_SPARSE}) {
        if (fp == QMC_FIRST_PASS_SPARSE && (!sparse_ok || k != QMC_KERNEL_AUTO)) continue;
        p.pass_kernel = k;
        p.first_pass = fp;
        const float ms = time_ms(st, [&] {
          return qmc_matmul(&p, A, lda, t, QMC_DTYPE_F32, out, ldo, nullptr, nullptr, st);
        }, 2, &rc);
        if (rc) return rc;
        if (ms < best.ms) best = TuneChoice{p.L1, k, fp, ms};
      }
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = best;
    tune_cache_append(key, best);
  }
  return apply_choice(p, best, t);
}

int autotune(Batch& b, const float* const* A, const int64_t* lda, float* const* out,
             const int64_t* ldo, cudaStream_t st) {
  int rc = QMC_OK;
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  for (size_t i = 0; i < b.plans.size(); ++i)
    if ((rc = tune_problem(*b.plans[i], b.t[i], A[i], lda[i], out[i], ldo[i], major * 10 + minor, st))) return rc;
  if (b.branches == 0) {
    float best = 1e30f;
    int best_n = 1;
    for (int n : {1, 2, 4, 8, 16}) {
      if (n > (int)b.br.size()) break;
      if ((rc = capture(b, A, lda, out, ldo, n))) return rc;
      const float ms = time_ms(st, [&] { return launch_graph(b, st); }, 3, &rc);
      if (rc) return rc;
      if (ms < best) { best = ms; best_n = n; }
    }
    b.branches = best_n;
  }
  b.tuned = true;
  return capture(b, A, lda, out, ldo, b.branches);
}

int run_graph(Batch& b, const float* const* A, const int64_t* lda, float* const* out,
              const int64_t* ldo, cudaStream_t st) {
  int rc;
  if (!b.tuned) {
    if ((rc = autotune(b, A, lda, out, ldo, st))) return rc;
  } else {
    const size_t n = b.plans.size();
    const bool same = b.exec && std::equal(A, A + n, b.keyA.begin()) && std::equal(out, out + n, b.keyOut.begin()) &&
                      std::equal(lda, lda + n, b.keyLda.begin()) && std::equal(ldo, ldo + n, b.keyLdo.begin());
    if (!same && (rc = capture(b, A, lda, out, ldo, b.branches))) return rc;
  }
  return launch_graph(b, st);
}

// Queue item(s) of one pass: the specialised tile loop where the pass has
// one in the queue (same conditions as the stand-alone launches), else the
// generic tile.
void queue_items(const Plan& p, const PassSpec& sp, int group, std::vector<BatchItem>& out) {
  const PassArgs& a = sp.a;
  const int npan = (a.T + 7) >> 3;
  const bool special = (p.pass_kernel == QMC_KERNEL_AUTO || p.pass_kernel == QMC_KERNEL_PIPELINED) &&
                       a.logW == 3 && !a.split && !a.a_f64;
  BatchItem it{};
  it.a = a;
  it.group = group;
  it.load = sp.load;
  it.store = sp.store;
  const bool gather768 = special && sp.load == LD_GATHER_A && sp.store == ST_SCRATCH && a.LP == 768 && a.fwd &&
                         !a.inv && !a.mul && a.twiddle < 0 && a.gp_em >= 1 && a.gp_em <= kGatherMax &&
                         (((uintptr_t)a.A) & 3u) == 0;
  const bool spec1024 = special && sp.load == LD_SCRATCH && sp.store == ST_SCRATCH && a.LP == 1024 && a.fwd &&
                        a.inv && a.mul == 1 && a.twiddle == 1 && a.point_stride == 1;
  const bool out768 = special && sp.load == LD_SCRATCH && sp.store == ST_OUT && a.LP == 768 && !a.fwd && a.inv &&
                      !a.mul && a.twiddle == 0 && !a.row_mean && !a.col_off && !a.out_exp && !a.exp_sum;
  constexpr int kChunk = 8;  // tiles per claim of the specialised loops
  if (gather768) {
    it.chunk = kChunk;
    if (a.lines) {
      const int nd = 2 * a.n_pair + a.n_direct;
      if (nd > 0) {
        it.kind = QK_DIRECT768;
        it.ntiles = nd * npan;
        out.push_back(it);
      }
      if (a.n_fft > 0) {
        it.kind = QK_GATHER768;
        it.ntiles = a.n_fft * npan;
        out.push_back(it);
      }
    } else {
      it.kind = QK_GATHER768;
      it.ntiles = a.n_linegroups * npan;
      out.push_back(it);
    }
    return;
  }
  if (spec1024 || out768) {
    it.kind = spec1024 ? QK_SPEC1024 : QK_OUT768;
    it.ntiles = a.n_linegroups * npan;
    it.chunk = kChunk;
    out.push_back(it);
    return;
  }
  // passes of length 256 in the register tile: the forward first pass, the
  // spectral pass, the un-permute pass, or the single pass of L = 256
  const bool fast_mode = (sp.load == LD_GATHER_A && sp.store == ST_SCRATCH && a.fwd && !a.inv && !a.mul) ||
                         (sp.load == LD_SCRATCH && sp.store == ST_SCRATCH && a.fwd && a.inv && a.mul) ||
                         (sp.load == LD_SCRATCH && sp.store == ST_OUT && !a.fwd && a.inv && !a.mul) ||
                         (sp.load == LD_GATHER_A && sp.store == ST_OUT && a.fwd && a.inv && a.mul);
  if (p.pass_kernel != QMC_KERNEL_GENERIC && a.LP == 256 && a.logW <= 3 && !a.split && !a.a_f64 && fast_mode) {
    it.kind = QK_FAST256;
    it.a.logV = 4 - a.logW;  // 16 lines: W columns x V line groups
    it.a.logM = 4;
    const int V = 1 << it.a.logV;
    it.gx = (a.n_linegroups + V - 1) / V;
    it.ntiles = it.gx * ((a.T + (1 << a.logW) - 1) >> a.logW);
    it.chunk = 8;
    out.push_back(it);
    return;
  }
  it.kind = QK_GENERIC;
  // two tiles per block (one per half) where two fit the queue's shared
  // memory budget, with fewer line groups per tile if needed; else one
  auto bytes = [](const PassArgs& x) { return (int)((generic_tile_smem(x) + 15) & ~(size_t)15); };
  PassArgs h = it.a;
  while (h.logV > 0 && 2 * (size_t)bytes(h) > kQueueSmemCap) {
    --h.logV;
    h.logM = h.logW + h.logV;
  }
  if (2 * (size_t)bytes(h) <= kQueueSmemCap) {
    it.a = h;
    it.teams = 2;
  } else {
    while (it.a.logV > 0 && (size_t)bytes(it.a) > kQueueSmemCap) {
      --it.a.logV;
      it.a.logM = it.a.logW + it.a.logV;
    }
    it.teams = 1;
  }
  it.sbytes = bytes(it.a);
  const int V = 1 << it.a.logV;
  it.gx = (a.n_linegroups + V - 1) / V;
  it.ntiles = it.gx * ((a.T + (1 << a.logW) - 1) >> a.logW);
  it.chunk = 8;
  out.push_back(it);
}

size_t item_smem(const BatchItem& it) {
  switch (it.kind) {
    case QK_DIRECT768: return kSmemDirect768;
    case QK_GATHER768: return kSmemGather768;
    case QK_SPEC1024: return kSmemSpec1024;
    case QK_OUT768: return kSmemOut768;
    case QK_PACK: return 0;
    case QK_SPARSE1024: return smem_sparse1024(it.a.n_linegroups);
    case QK_FAST256: return sizeof(cx<float>) * (256 + (256 + 16) * 16);
  }
  return (size_t)it.teams * it.sbytes;
}

// Stage k (0..2) items of one problem.  A problem whose forward product
// takes the sparse first pass with a 1024-point spectral pass packs its
// rows in stage 0 and sums the spectral pass's lines from them in stage 1.
void problem_items(const Plan& p, const std::vector<PassSpec>& specs, const PassArgs* sparse, int k, int group,
                   std::vector<BatchItem>& out) {
  if (sparse && k < 2) {
    BatchItem it{};
    it.a = *sparse;
    it.group = group;
    it.kind = k == 0 ? QK_PACK : QK_SPARSE1024;
    it.ntiles = k == 0 ? sparse->sp_s : sparse->n_linegroups * ((sparse->T + 7) >> 3);
    it.chunk = k == 0 ? 16 : 8;
    out.push_back(it);
    return;
  }
  queue_items(p, specs[k], group, out);
}

int run_persistent(Batch& b, const float* const* A, const int64_t* lda, float* const* out,
                   const int64_t* ldo, cudaStream_t st) {
  int rc;
  const int np = (int)b.plans.size();
  std::vector<std::vector<PassSpec>> specs(np);
  std::vector<PassArgs> sparse(np);
  std::vector<char> has_sparse(np, 0);
  std::vector<ColstatsJob> jobs(np);
  // column statistics (row 0, scales) per problem, then the pass list
  int partial_blocks = 0, final_blocks = 0;
  for (int i = 0; i < np; ++i) {
    Plan& p = *b.plans[i];
    PassArgs base;
    if ((rc = forward_prologue(p, A[i], lda[i], b.t[i], QMC_DTYPE_F32, out[i], ldo[i], st, &base, &jobs[i])))
      return rc;
    jobs[i].blk_partial = partial_blocks;
    jobs[i].blk_final = final_blocks;
    partial_blocks += jobs[i].blocks_partial;
    final_blocks += jobs[i].blocks_final;
    PassSpec sp[3];
    int n = 0;
    if ((rc = product_passes(p, +1, base, sp, &n))) return rc;
    specs[i].assign(sp, sp + n);
    PassArgs sb;
    if (sparse_spectral_args(p, +1, sp, n, &sb) && sb.LP == 1024 && !sb.split && !sb.a_f64 &&
        sb.n_linegroups <= 1024 && (int64_t)sb.n_linegroups * sb.LP == sb.L) {
      sparse[i] = sb;
      has_sparse[i] = 1;
    }
  }
  // stage-major items; within a stage the largest problems first
  std::vector<int> order(np);
  for (int i = 0; i < np; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (double)b.plans[x]->L * b.t[x] > (double)b.plans[y]->L * b.t[y];
  });
  b.h_items.clear();
  const int ngroups = np * 3;
  std::vector<int> group_chunks(ngroups, 0);
  size_t smem = 0;
  for (int k = 0; k < 3; ++k) {
    for (int i : order) {
      if (k >= (int)specs[i].size()) continue;
      const size_t first = b.h_items.size();
      problem_items(*b.plans[i], specs[i], has_sparse[i] ? &sparse[i] : nullptr, k, i * 3 + k, b.h_items);
      for (size_t q = first; q < b.h_items.size(); ++q) {
        BatchItem& it = b.h_items[q];
        it.dep = k > 0 ? i * 3 + k - 1 : -1;
        group_chunks[it.group] += (it.ntiles + it.chunk - 1) / it.chunk;
        smem = std::max(smem, item_smem(it));
      }
    }
  }
  const int nitems = (int)b.h_items.size();
  b.h_chunk_item.clear();
  for (int q = 0; q < nitems; ++q) {
    BatchItem& it = b.h_items[q];
    it.need = it.dep >= 0 ? group_chunks[it.dep] : 0;
    if (q == b.test_block_item && it.dep >= 0) it.need += 1;  // never reached
    it.first = (int)b.h_chunk_item.size();
    it.nchunks = (it.ntiles + it.chunk - 1) / it.chunk;
    b.h_chunk_item.insert(b.h_chunk_item.end(), it.nchunks, q);
  }
  const int total = (int)b.h_chunk_item.size();
  const int cap_counters = ngroups + 1;
  if (cap_counters > b.cap_counters) {
    cudaFree(b.d_counters);
    b.d_counters = nullptr;
    b.cap_counters = 0;
    if (cudaMalloc(&b.d_counters, sizeof(int) * cap_counters) != cudaSuccess) {
      cudaGetLastError();
      return QMC_ERR_ALLOC;
    }
    b.cap_counters = cap_counters;
  }
  // blob: items | jobs | chunk items, each at a 256-byte offset
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t off_jobs = up(sizeof(BatchItem) * nitems);
  const size_t off_chunks = off_jobs + up(sizeof(ColstatsJob) * np);
  const size_t bytes = off_chunks + sizeof(int) * (size_t)total;
  std::vector<unsigned char> blob(bytes, 0);
  memcpy(blob.data(), b.h_items.data(), sizeof(BatchItem) * nitems);
  memcpy(blob.data() + off_jobs, jobs.data(), sizeof(ColstatsJob) * np);
  memcpy(blob.data() + off_chunks, b.h_chunk_item.data(), sizeof(int) * (size_t)total);
  // the previous launch reads the blob and the counters: a call on another
  // stream starts after it
  if (b.done_ev && cudaStreamWaitEvent(st, b.done_ev, 0) != cudaSuccess) {
    cudaGetLastError();
    return QMC_ERR_CUDA;
  }
  if (blob != b.last_blob) {
    if (b.up_ev && cudaEventSynchronize(b.up_ev) != cudaSuccess) return QMC_ERR_CUDA;  // h_stage free again
    if (bytes > b.cap_blob) {
      if (b.d_blob) { cudaFree(b.d_blob); b.d_blob = nullptr; }
      if (b.h_stage) { cudaFreeHost(b.h_stage); b.h_stage = nullptr; }
      b.cap_blob = 0;
      b.last_blob.clear();
      if (cudaMalloc(&b.d_blob, bytes) != cudaSuccess || cudaMallocHost(&b.h_stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        return QMC_ERR_ALLOC;
      }
      b.cap_blob = bytes;
    }
    if (!b.up_ev && cudaEventCreateWithFlags(&b.up_ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return QMC_ERR_CUDA;
    }
    memcpy(b.h_stage, blob.data(), bytes);
    if (cudaMemcpyAsync(b.d_blob, b.h_stage, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaEventRecord(b.up_ev, st) != cudaSuccess) {
      cudaGetLastError();
      b.last_blob.clear();
      return QMC_ERR_CUDA;
    }
    b.last_blob.swap(blob);
  }
  const BatchItem* d_items = reinterpret_cast<const BatchItem*>(b.d_blob);
  const ColstatsJob* d_jobs = reinterpret_cast<const ColstatsJob*>(b.d_blob + off_jobs);
  const int* d_chunk_item = reinterpret_cast<const int*>(b.d_blob + off_chunks);
  if ((rc = launch_colstats_multi(d_jobs, np, partial_blocks, final_blocks, st))) return rc;
  if (total < 1) return QMC_OK;
  cudaMemsetAsync(b.d_counters, 0, sizeof(int) * cap_counters, st);
  static KernelSetup setup;
  int grid = 0;
  if ((rc = setup_kernel(k_batch, setup, smem, kQueueThreads, &grid))) return rc;
  int dev = 0, clock_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
  grid = std::min(grid, total);
  const long long wait_cycles = (long long)b.wait_us * (long long)(clock_khz > 0 ? clock_khz : 2000000) / 1000;
  k_batch<<<grid, kQueueThreads, smem, st>>>(d_items, d_chunk_item, total, b.d_counters,
                                             b.d_counters + ngroups, b.d_err, wait_cycles);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
  if (!b.done_ev && cudaEventCreateWithFlags(&b.done_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return QMC_ERR_CUDA;
  }
  return cudaEventRecord(b.done_ev, st) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

void destroy(Batch* b) {
  if (!b) return;
  free_graph(*b);
  for (auto s : b->br) cudaStreamDestroy(s);
  for (auto e : b->ev) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->d_blob); cudaFree(b->d_counters); cudaFree(b->d_err);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->up_ev) cudaEventDestroy(b->up_ev);
  if (b->done_ev) cudaEventDestroy(b->done_ev);
  delete b;
}

}  // namespace

extern "C" {

int qmc_batch_create(void** batch, void* const* plans, const int32_t* t_host, int32_t count,
                     void* stream) {
  if (!batch || !plans || !t_host || count < 1) return QMC_ERR_INVALID;
  *batch = nullptr;
  Batch* b = new (std::nothrow) Batch();
  if (!b) return QMC_ERR_ALLOC;
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || t_host[i] < 1) { destroy(b); return QMC_ERR_INVALID; }
    if (static_cast<Plan*>(plans[i])->pset) { destroy(b); return QMC_ERR_UNSUPPORTED; }
    b->plans.push_back(static_cast<Plan*>(plans[i]));
    b->t.push_back(t_host[i]);
    const int rc = qmc_plan_reserve(plans[i], t_host[i]);
    if (rc) { destroy(b); return rc; }
  }
  const int nbr = 16;
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&b->d_err, sizeof(int)) == cudaSuccess &&
            cudaMemset(b->d_err, 0, sizeof(int)) == cudaSuccess;
  for (int k = 0; ok && k < nbr; ++k) {
    cudaStream_t s;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->br.push_back(s);
  }
  for (int k = 0; ok && k < nbr + 1; ++k) {
    cudaEvent_t e;
    ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->ev.push_back(e);
  }
  if (!ok) { cudaGetLastError(); destroy(b); return QMC_ERR_CUDA; }
  (void)stream;
  *batch = b;
  return QMC_OK;
}

int qmc_batch_set_option(void* batch, int32_t option, int64_t value) {
  if (!batch) return QMC_ERR_INVALID;
  Batch& b = *static_cast<Batch*>(batch);
  switch (option) {
    case QMC_BATCH_OPT_MODE:
      if (value != QMC_BATCH_GRAPH && value != QMC_BATCH_PERSISTENT) return QMC_ERR_INVALID;
      b.mode = (int)value;
      return QMC_OK;
    case QMC_BATCH_OPT_BRANCHES:
      if (value < 0 || value > (int64_t)b.br.size()) return QMC_ERR_INVALID;
      b.branches = (int)value;
      b.tuned = value != 0 && b.tuned;
      free_graph(b);
      return QMC_OK;
    case QMC_BATCH_OPT_WAIT_LIMIT_US:
      if (value < 1) return QMC_ERR_INVALID;
      b.wait_us = value;
      return QMC_OK;
    case QMC_BATCH_OPT_TEST_BLOCK_ITEM:
      b.test_block_item = (int)value;
      return QMC_OK;
  }
  return QMC_ERR_INVALID;
}

int qmc_batch_matmul(void* batch, const float* const* A, const int64_t* lda, float* const* out,
                     const int64_t* ldo, void* stream) {
  if (!batch || !A || !lda || !out || !ldo) return QMC_ERR_INVALID;
  Batch& b = *static_cast<Batch*>(batch);
  for (size_t i = 0; i < b.plans.size(); ++i)
    if (!A[i] || !out[i] || lda[i] < b.t[i] || ldo[i] < b.t[i]) return QMC_ERR_SHAPE;
  cudaStream_t st = (cudaStream_t)stream;
  return b.mode == QMC_BATCH_PERSISTENT ? run_persistent(b, A, lda, out, ldo, st)
                                        : run_graph(b, A, lda, out, ldo, st);
}

int qmc_batch_sync_status(void* batch, void* stream) {
  if (!batch) return QMC_ERR_INVALID;
  Batch& b = *static_cast<Batch*>(batch);
  int h = 0;
  if (cudaMemcpyAsync(&h, b.d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return QMC_ERR_CUDA;
  if (!h) return QMC_OK;
  cudaMemsetAsync(b.d_err, 0, sizeof(int), (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  return (h & kErrTimeout) ? QMC_ERR_TIMEOUT : QMC_ERR_DEVICE;
}

int qmc_batch_destroy(void* batch) {
  if (!batch) return QMC_ERR_INVALID;
  cudaDeviceSynchronize();
  destroy(static_cast<Batch*>(batch));
  return QMC_OK;
}

}  // extern "C"
