// Batched stepping of many independent lattices of uneven sizes.
//
// Work unit: a tile of 32 rows x TX columns of one lattice, one warp per column, processed
// by one block (TX = warps per block, the autotuned tile width).  All lattices of a batch
// are laid end to end in one tile index space (prefix sums in BatchLattice::tile_begin, y
// fastest inside a lattice) and a device table gives each tile's lattice, so everything a
// block reads about its lattice is uniform across the block.  Each warp runs the same strip
// step as the single-lattice kernels (step_fp64.cuh / step_fp32.cuh), so results are
// bit-identical to lbm_run per lattice (all three forms: FP64, FP64 with the fixed-point
// relaxation, whose blocks stage their strips in dynamic shared memory, and FP32).
//
// Modes:
//   LBM_BATCH_PER_STEP   one launch per step over all tiles of all lattices;
//   LBM_BATCH_PERSISTENT one cooperative launch for all steps: blocks stride over the
//                        tiles, and a grid barrier separates steps.  The barrier's wait is
//                        bounded in time; on expiry it sets an error word, every block
//                        returns, and lbm_batch_status reports LBM_ETIMEOUT.  Loads inside
//                        this kernel bypass L1 (the sources were written by other SMs
//                        earlier in the same launch);
//   LBM_BATCH_LOOP       the plain single-lattice kernel launched per lattice per step
//                        (the comparison baseline).
// The autotuner times candidate (mode, tile width, blocks per SM) on the batch itself
// and keeps the fastest, in the spirit of the paper's start-up mini-benchmarks that pick
// its tuning parameters (Sec. 6).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/lbm_d2q37.h"
#include "kernels.h"
#include "step_fix64.cuh"
#include "step_fp32.cuh"

namespace d2q37 {

struct BatchLattice {
  StepArgs a;
  void* f[2];            // state buffers; f[parity] holds the current state
  long long tile_begin;  // first tile of this lattice in the batch index space
  int tiles_y;           // ceil(ly / 32)
  int tiles_x;           // ceil(lx / TX)
};

// The first three words are reset by every persistent launch; `sticky` is not.
struct BatchSync {
  unsigned int arrived;  // grid-barrier arrivals since the launch started
  unsigned int error;    // 1 after a barrier wait of this launch expired (stops every block)
  unsigned int step;     // step whose barrier expired
  unsigned int sticky;   // 1 after any launch's wait expired, until lbm_batch_status reads it
};
constexpr size_t kBatchSyncLaunchBytes = 3 * sizeof(unsigned int);

namespace {

// Step kinds: the strip functions of the three storage/arithmetic forms.
// kFp32Scaled: FP32 storage where some lattice has a reference density of 2 or more (the
// moment sums read each lattice's scale constants; see step_fp32.cuh); kFp32Cons and
// kFp32ConsScaled: the same with the conserved-moment correction (LBM_FP32_CONSERVED).
enum BatchKind { kFp64 = 0, kFp32 = 1, kFix64 = 2, kFp32Scaled = 3, kFp32Cons = 4, kFp32ConsScaled = 5 };
constexpr bool kind_fp32(int k) { return k == kFp32 || k == kFp32Scaled || k == kFp32Cons || k == kFp32ConsScaled; }

template <int K>
struct KindOf {
  using T = double;
};
template <>
struct KindOf<kFp32> {
  using T = float;
};
template <>
struct KindOf<kFp32Scaled> {
  using T = float;
};
template <>
struct KindOf<kFp32Cons> {
  using T = float;
};
template <>
struct KindOf<kFp32ConsScaled> {
  using T = float;
};

// Shared memory of a block: the fixed-point form stages 37 x 32 doubles per warp.
inline size_t batch_smem_bytes(int kind, int warps) {
  return kind == kFix64 ? (size_t)warps * Q * 32 * sizeof(double) : 0;
}

// Tile t of the batch (32 rows x TX columns, one warp per column, as the single-lattice
// kernels): its lattice comes from a per-tile table, so everything that depends on the
// lattice is uniform across the block.
template <int KIND, bool PERIODIC, class Ld>
__device__ __forceinline__ void batch_tile(const BatchLattice* __restrict__ L, const unsigned short* __restrict__ tl,
                                           long long t, int parity, Ld ld, double* staged) {
  using T = typename KindOf<KIND>::T;
  const int j = tl[t];
  const BatchLattice& B = L[j];
  const long long local = t - B.tile_begin;
  const int tx = (int)(local / B.tiles_y);
  const int ty = (int)(local - (long long)tx * B.tiles_y);
  const int x = tx * (int)blockDim.y + (int)threadIdx.y;
  if (x >= B.a.lx) return;  // uniform per warp
  const T* src = (const T*)B.f[parity];
  T* dst = (T*)B.f[parity ^ 1];
  if constexpr (KIND == kFp64) step_strip_fp64<PERIODIC>(src, dst, B.a, B.a, x, ty * 32, ld);
  else if constexpr (KIND == kFix64)
    step_strip_fix64<PERIODIC>(src, dst, B.a, B.a, x, ty * 32, ld, staged + threadIdx.y * (Q * 32));
  else
    step_strip_fp32<PERIODIC, KIND == kFp32Scaled || KIND == kFp32ConsScaled, KIND == kFp32Cons || KIND == kFp32ConsScaled>(
        src, dst, B.a, B.a, x, ty * 32, ld);
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier with a bounded wait.  Returns false (for every thread of the block) when
// the wait expired here or in another block.
__device__ __forceinline__ bool grid_barrier(BatchSync* sync, unsigned target, long long timeout_ns, int step) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    atomicAdd(&sync->arrived, 1u);
    const unsigned long long t0 = global_ns();
    const long long max_iter = timeout_ns / 64 + 4096;  // also bounded by iterations
    long long it = 0;
    int ok = 1;
    while (ld_acquire_gpu(&sync->arrived) < target) {
      if (ld_acquire_gpu(&sync->error) != 0u) {
        ok = 0;
        break;
      }
      if ((long long)(global_ns() - t0) > timeout_ns || ++it > max_iter) {
        if (atomicCAS(&sync->error, 0u, 1u) == 0u) atomicExch(&sync->step, (unsigned)step);
        atomicExch(&sync->sticky, 1u);
        ok = 0;
        break;
      }
      __nanosleep(128);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace

// Register caps, with at most 256 threads per block (8 warps): the FP32 step keeps three
// such blocks resident per SM (80 registers), the float64 step two (128 registers, as its
// single-lattice kernel), the fixed-point FP64 step and the conserved-moment FP32 step the
// 96 registers of their single-lattice kernels (5 blocks of 4 warps per SM).
constexpr int batch_max_regs(int kind) {
  return kind == kFp64 ? 128 : (kind == kFix64 || kind == kFp32Cons || kind == kFp32ConsScaled ? 96 : 80);
}

extern __shared__ double batch_staged[];

template <int KIND, bool PERIODIC>
__global__ void __launch_bounds__(256) __maxnreg__(batch_max_regs(KIND)) k_batch_step(const BatchLattice* __restrict__ L,
                                                    const unsigned short* __restrict__ tl, long long total,
                                                    int parity) {
  const long long t = blockIdx.x;
  if (t >= total) return;
  batch_tile<KIND, PERIODIC>(L, tl, t, parity, LdReadOnly(), batch_staged);
}

template <int KIND, bool PERIODIC>
__global__ void __launch_bounds__(256) __maxnreg__(batch_max_regs(KIND)) k_batch_persistent(const BatchLattice* __restrict__ L,
                                                          const unsigned short* __restrict__ tl, long long total,
                                                          int parity0, int steps, BatchSync* sync, unsigned phantom,
                                                          long long timeout_ns) {
  for (int st = 0; st < steps; ++st) {
    const int parity = (parity0 + st) & 1;
    for (long long t = blockIdx.x; t < total; t += gridDim.x)
      batch_tile<KIND, PERIODIC>(L, tl, t, parity, LdL2(), batch_staged);
    if (st + 1 < steps && !grid_barrier(sync, (unsigned)(st + 1) * gridDim.x + phantom, timeout_ns, st)) return;
  }
}

}  // namespace d2q37

using namespace d2q37;

struct lbm_batch {
  int n = 0;
  int precision = LBM_FP64;
  int periodic = 0;
  int fp32_scaled = 0;  // FP32 batch with some reference density of 2 or more
  long long total_tiles = 0;
  unsigned short* dev_tile_lattice = nullptr;  // lattice of every tile
  size_t tile_table_cap = 0;
  std::vector<BatchLattice> host;
  BatchLattice* dev_lattices = nullptr;
  BatchSync* dev_sync = nullptr;
  int parity = 0;
  int mode = LBM_BATCH_PER_STEP;
  int warps_per_block = 4;  // = tile width TX
  int blocks_per_sm = 0;  // 0 = as many as fit
  long long timeout_ns = 2000000000LL;
  unsigned phantom = 0;
  int device = 0;
  int sms = 0;
};

namespace {

thread_local int32_t g_batch_cuda_error = 0;

int32_t cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  g_batch_cuda_error = (int32_t)e;
  return LBM_ECUDA;
}

int kind_of(const lbm_batch* b) {
  if (b->precision == LBM_FP32_SHIFTED) return b->fp32_scaled ? kFp32Scaled : kFp32;
  if (b->precision == LBM_FP32_CONSERVED) return b->fp32_scaled ? kFp32ConsScaled : kFp32Cons;
  return b->precision == LBM_FP64_FIXED ? kFix64 : kFp64;
}

template <int K>
void* persistent_fn(bool periodic) {
  return periodic ? (void*)k_batch_persistent<K, true> : (void*)k_batch_persistent<K, false>;
}
template <int K>
void* per_step_fn(bool periodic) {
  return periodic ? (void*)k_batch_step<K, true> : (void*)k_batch_step<K, false>;
}

void* persistent_kernel(const lbm_batch* b) {
  switch (kind_of(b)) {
    case kFix64: return persistent_fn<kFix64>(b->periodic);
    case kFp32: return persistent_fn<kFp32>(b->periodic);
    case kFp32Scaled: return persistent_fn<kFp32Scaled>(b->periodic);
    case kFp32Cons: return persistent_fn<kFp32Cons>(b->periodic);
    case kFp32ConsScaled: return persistent_fn<kFp32ConsScaled>(b->periodic);
    default: return persistent_fn<kFp64>(b->periodic);
  }
}
void* per_step_kernel(const lbm_batch* b) {
  switch (kind_of(b)) {
    case kFix64: return per_step_fn<kFix64>(b->periodic);
    case kFp32: return per_step_fn<kFp32>(b->periodic);
    case kFp32Scaled: return per_step_fn<kFp32Scaled>(b->periodic);
    case kFp32Cons: return per_step_fn<kFp32Cons>(b->periodic);
    case kFp32ConsScaled: return per_step_fn<kFp32ConsScaled>(b->periodic);
    default: return per_step_fn<kFp64>(b->periodic);
  }
}

// Raises both kernels' dynamic shared memory limit to the largest staging a block can
// need (8 warps); called once per plan.
int32_t allow_batch_smem(const lbm_batch* b) {
  const size_t smem = batch_smem_bytes(kind_of(b), 8);
  if (smem <= 48 * 1024) return LBM_OK;
  if (cudaFuncSetAttribute(persistent_kernel(b), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(per_step_kernel(b), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return cuda_status(cudaGetLastError());
  return LBM_OK;
}

// Blocks of wpb warps that fit on one SM for the persistent kernel.
int max_blocks_per_sm(const lbm_batch* b, int wpb) {
  const size_t smem = batch_smem_bytes(kind_of(b), wpb);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persistent_kernel(b), 32 * wpb, smem) != cudaSuccess)
    return 0;
  return nb;
}

int32_t launch_per_step(lbm_batch* b, int steps, cudaStream_t s) {
  if (b->total_tiles > 0x7fffffffLL) return LBM_EINVAL;
  const size_t smem = batch_smem_bytes(kind_of(b), b->warps_per_block);
  const BatchLattice* L = b->dev_lattices;
  const unsigned short* tl = b->dev_tile_lattice;
  long long total = b->total_tiles;
  for (int st = 0; st < steps; ++st) {
    int par = (b->parity + st) & 1;
    void* args[] = {(void*)&L, (void*)&tl, &total, &par};
    const int32_t st_ = cuda_status(cudaLaunchKernel(per_step_kernel(b), dim3((unsigned)total),
                                                     dim3(32, b->warps_per_block), args, smem, s));
    if (st_ != LBM_OK) return st_;
  }
  return LBM_OK;
}

int32_t launch_persistent(lbm_batch* b, int steps, cudaStream_t s) {
  const int wpb = b->warps_per_block;
  const int fit = max_blocks_per_sm(b, wpb);
  if (fit <= 0) return LBM_EINVAL;
  const int per_sm = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, fit) : fit;
  const unsigned grid = (unsigned)(per_sm * b->sms);
  if ((unsigned long long)steps * grid + b->phantom >= 0x7fffffffULL) return LBM_EINVAL;
  int32_t st = cuda_status(cudaMemsetAsync(b->dev_sync, 0, kBatchSyncLaunchBytes, s));
  if (st != LBM_OK) return st;
  const BatchLattice* L = b->dev_lattices;
  const unsigned short* tl = b->dev_tile_lattice;
  long long total = b->total_tiles;
  int parity0 = b->parity;
  BatchSync* sync = b->dev_sync;
  unsigned phantom = b->phantom;
  long long timeout = b->timeout_ns;
  void* args[] = {(void*)&L, (void*)&tl, &total, &parity0, &steps, &sync, &phantom, &timeout};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32, wpb);
  cfg.dynamicSmemBytes = batch_smem_bytes(kind_of(b), wpb);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cuda_status(cudaLaunchKernelExC(&cfg, persistent_kernel(b), args));
}

int32_t launch_loop(lbm_batch* b, int steps, cudaStream_t s) {
  for (int st = 0; st < steps; ++st) {
    const int par = (b->parity + st) & 1;
    for (int j = 0; j < b->n; ++j) {
      const BatchLattice& B = b->host[j];
      const int32_t r = cuda_status(launch_step(B.f[par], B.f[par ^ 1], B.a, b->precision, s));
      if (r != LBM_OK) return r;
    }
  }
  return LBM_OK;
}

int32_t run(lbm_batch* b, int steps, cudaStream_t s) {
  if (steps <= 0) return steps == 0 ? LBM_OK : LBM_EINVAL;
  int32_t st;
  switch (b->mode) {
    case LBM_BATCH_PER_STEP: st = launch_per_step(b, steps, s); break;
    case LBM_BATCH_PERSISTENT: st = launch_persistent(b, steps, s); break;
    case LBM_BATCH_LOOP: st = launch_loop(b, steps, s); break;
    default: return LBM_EINVAL;
  }
  if (st == LBM_OK) b->parity ^= (steps & 1);
  return st;
}

// Tile layout for tiles of 32 rows x tx columns, and the per-tile lattice table, uploaded
// to the device (synchronous; grows the table allocation when needed).
int32_t relayout(lbm_batch* b, int tx) {
  long long tiles = 0;
  for (BatchLattice& L : b->host) {
    L.tiles_y = (L.a.ly + 31) / 32;
    L.tiles_x = (L.a.lx + tx - 1) / tx;
    L.tile_begin = tiles;
    tiles += (long long)L.tiles_y * L.tiles_x;
  }
  std::vector<unsigned short> table((size_t)tiles);
  for (int j = 0; j < b->n; ++j) {
    const BatchLattice& L = b->host[j];
    std::fill(table.begin() + L.tile_begin, table.begin() + L.tile_begin + (long long)L.tiles_y * L.tiles_x,
              (unsigned short)j);
  }
  if ((size_t)tiles > b->tile_table_cap) {
    if (b->dev_tile_lattice) cudaFree(b->dev_tile_lattice);
    b->dev_tile_lattice = nullptr;
    b->tile_table_cap = 0;
    if (cudaMalloc(&b->dev_tile_lattice, sizeof(unsigned short) * (size_t)tiles) != cudaSuccess) return LBM_ENOMEM;
    b->tile_table_cap = (size_t)tiles;
  }
  b->total_tiles = tiles;
  b->warps_per_block = tx;
  int32_t st = cuda_status(cudaMemcpy(b->dev_tile_lattice, table.data(), sizeof(unsigned short) * (size_t)tiles,
                                      cudaMemcpyHostToDevice));
  if (st != LBM_OK) return st;
  return cuda_status(cudaMemcpy(b->dev_lattices, b->host.data(), sizeof(BatchLattice) * b->n, cudaMemcpyHostToDevice));
}

bool overlap(const void* a, const void* b, int64_t bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + (uintptr_t)bytes && y < x + (uintptr_t)bytes;
}

}  // namespace

extern "C" {

int32_t lbm_batch_plan(const lbm_params* params, void* const* f_a, void* const* f_b, int32_t n, lbm_batch** out) {
  if (!params || !f_a || !f_b || !out || n <= 0 || n > 65535) return LBM_EINVAL;
  *out = nullptr;
  lbm_batch* b = new lbm_batch();
  b->n = n;
  b->precision = params[0].precision;
  b->periodic = params[0].bc == LBM_BC_PERIODIC_Y;
  for (int j = 0; j < n; ++j) {
    const lbm_params* p = &params[j];
    const int64_t bytes = lbm_buffer_bytes(p);
    if (!params_valid(p) || p->precision != b->precision || p->bc != params[0].bc || bytes <= 0 || !f_a[j] ||
        !f_b[j] || ((uintptr_t)f_a[j] % 16) || ((uintptr_t)f_b[j] % 16) || overlap(f_a[j], f_b[j], bytes)) {
      delete b;
      return LBM_EINVAL;
    }
    BatchLattice L;
    memset(&L, 0, sizeof(L));
    L.a = make_step_args(p);
    if (L.a.fix_back != 1.0 / 4503599627370496.0) b->fp32_scaled = 1;
    L.f[0] = f_a[j];
    L.f[1] = f_b[j];
    b->host.push_back(L);
  }
  // no two of the 2n state buffers may overlap (a step reads one lattice's buffer while
  // other blocks write another's)
  {
    std::vector<std::pair<uintptr_t, uintptr_t>> ranges;
    for (int j = 0; j < n; ++j) {
      const uintptr_t bytes = (uintptr_t)lbm_buffer_bytes(&params[j]);
      ranges.push_back({(uintptr_t)f_a[j], (uintptr_t)f_a[j] + bytes});
      ranges.push_back({(uintptr_t)f_b[j], (uintptr_t)f_b[j] + bytes});
    }
    std::sort(ranges.begin(), ranges.end());
    for (size_t k = 1; k < ranges.size(); ++k)
      if (ranges[k].first < ranges[k - 1].second) {
        delete b;
        return LBM_EINVAL;
      }
  }
  cudaDeviceProp prop;
  if (cudaGetDevice(&b->device) != cudaSuccess || cudaGetDeviceProperties(&prop, b->device) != cudaSuccess) {
    delete b;
    return LBM_ECUDA;
  }
  b->sms = prop.multiProcessorCount;
  if (cudaMalloc(&b->dev_lattices, sizeof(BatchLattice) * n) != cudaSuccess) {
    delete b;
    return LBM_ENOMEM;
  }
  if (cudaMalloc(&b->dev_sync, sizeof(BatchSync)) != cudaSuccess) {
    cudaFree(b->dev_lattices);
    delete b;
    return LBM_ENOMEM;
  }
  if (relayout(b, 4) != LBM_OK || cudaMemset(b->dev_sync, 0, sizeof(BatchSync)) != cudaSuccess ||
      allow_batch_smem(b) != LBM_OK) {
    cudaFree(b->dev_tile_lattice);
    cudaFree(b->dev_lattices);
    cudaFree(b->dev_sync);
    delete b;
    return LBM_ECUDA;
  }
  *out = b;
  return LBM_OK;
}

int32_t lbm_batch_configure(lbm_batch* b, int32_t mode, int32_t tile_columns, int32_t blocks_per_sm) {
  if (!b || (mode != LBM_BATCH_PER_STEP && mode != LBM_BATCH_PERSISTENT && mode != LBM_BATCH_LOOP)) return LBM_EINVAL;
  if (tile_columns != 1 && tile_columns != 2 && tile_columns != 4 && tile_columns != 8) return LBM_EINVAL;
  if (blocks_per_sm < 0 || blocks_per_sm > 64) return LBM_EINVAL;
  b->mode = mode;
  b->blocks_per_sm = blocks_per_sm;
  if (tile_columns != b->warps_per_block) return relayout(b, tile_columns);
  return LBM_OK;
}

int32_t lbm_batch_config(const lbm_batch* b, int32_t* mode, int32_t* tile_columns, int32_t* blocks_per_sm) {
  if (!b) return LBM_EINVAL;
  if (mode) *mode = b->mode;
  if (tile_columns) *tile_columns = b->warps_per_block;
  if (blocks_per_sm) {
    const int fit = b->mode == LBM_BATCH_PERSISTENT ? max_blocks_per_sm(b, b->warps_per_block) : 0;
    *blocks_per_sm = b->mode == LBM_BATCH_PERSISTENT ? (b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, fit) : fit)
                                                      : 0;
  }
  return LBM_OK;
}

int32_t lbm_batch_set_wait(lbm_batch* b, int64_t timeout_ns, int32_t phantom_arrivals) {
  if (!b || timeout_ns <= 0 || timeout_ns > 60LL * 1000000000LL || phantom_arrivals < 0) return LBM_EINVAL;
  b->timeout_ns = timeout_ns;
  b->phantom = (unsigned)phantom_arrivals;
  return LBM_OK;
}

int32_t lbm_batch_run(lbm_batch* b, int32_t n_steps, void* stream) {
  if (!b || n_steps < 0) return LBM_EINVAL;
  return run(b, n_steps, (cudaStream_t)stream);
}

// Batches up to this many sites also try the persistent launch when autotuning.
constexpr int64_t kPersistentCandidateSites = 1 << 20;

int32_t lbm_batch_autotune(lbm_batch* b, int32_t trial_steps, void* stream) {
  if (!b || trial_steps < 1) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  struct Cand {
    int mode, tx, bps;
  };
  std::vector<Cand> cands;
  for (int tx : {2, 4, 8}) cands.push_back({LBM_BATCH_PER_STEP, tx, 0});
  // The persistent launch saves one kernel boundary per step (a few microseconds) but its
  // loads must bypass L1 (other SMs rewrite the buffers between steps), which measured
  // 7 % (float64) to 32 % (FP32) slower per step on batches of millions of sites.  It is
  // a candidate only where a step is short enough for the boundary to matter.
  if (lbm_batch_sites(b) <= kPersistentCandidateSites) {
    for (int tx : {2, 4, 8}) {
      const int fit = max_blocks_per_sm(b, tx);
      for (int bps = fit; bps >= 1 && bps >= fit - 1; --bps) cands.push_back({LBM_BATCH_PERSISTENT, tx, bps});
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LBM_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LBM_ECUDA;
  }
  float best = 1e30f;
  Cand best_c = {b->mode, b->warps_per_block, b->blocks_per_sm};
  int32_t st = LBM_OK;
  for (const Cand& c : cands) {
    if ((st = lbm_batch_configure(b, c.mode, c.tx, c.bps)) != LBM_OK) break;
    if ((st = run(b, 1, s)) != LBM_OK) break;  // warm-up
    cudaEventRecord(e0, s);
    if ((st = run(b, trial_steps, s)) != LBM_OK) break;
    cudaEventRecord(e1, s);
    if ((st = cuda_status(cudaEventSynchronize(e1))) != LBM_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int32_t st2 = lbm_batch_configure(b, best_c.mode, best_c.tx, best_c.bps);
  return st != LBM_OK ? st : st2;
}

int32_t lbm_batch_parity(const lbm_batch* b) { return b ? b->parity : -1; }

int32_t lbm_batch_status(lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  BatchSync h;
  const int32_t st = cuda_status(cudaMemcpy(&h, b->dev_sync, sizeof(h), cudaMemcpyDeviceToHost));
  if (st != LBM_OK) return st;
  if (h.sticky) {
    cudaMemset(b->dev_sync, 0, sizeof(BatchSync));
    return LBM_ETIMEOUT;
  }
  return LBM_OK;
}

int64_t lbm_batch_sites(const lbm_batch* b) {
  if (!b) return -1;
  int64_t s = 0;
  for (const BatchLattice& L : b->host) s += (int64_t)L.a.lx * L.a.ly;
  return s;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaFree(b->dev_tile_lattice);
  cudaFree(b->dev_lattices);
  cudaFree(b->dev_sync);
  delete b;
}

}  // extern "C"
