// persistent.cuh -- the persistent forms (TILE, GRID, GRID with activity-aware
// evaluation) and the table of their compiled launch-bounds variants.
//
//   TILE   each CTA takes a tile of lanes (instances) from an atomic queue,
//          longest remaining work first, and walks every layer of every cycle
//          of that tile with CTA barriers only (instances are independent).
//   GRID   the whole grid walks each layer for all lanes, separated by a
//          software grid barrier with a bounded wait.
#pragma once
#include <cstddef>
#include <cstdint>

#include "kernels.cuh"

namespace rteaal {

struct TileArgs {
  uint32_t* counter;             // scratch: next queue position
  const uint32_t* order;         // queue position -> tile (longest first), null = identity
  const uint32_t* tile_cycles;   // per tile, null -> uniform
  uint32_t n_tiles, tile_lanes;
  FastDiv tpo;                   // tile_lanes / V
};

template <int V, int U, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_tile(DDesign d, DSim s, TileArgs t) {
  __shared__ uint32_t sh_q;
  for (;;) {
    if (threadIdx.x == 0) sh_q = atomicAdd(t.counter, 1u);
    __syncthreads();
    const uint32_t q = sh_q;
    __syncthreads();
    if (q >= t.n_tiles) return;
    const uint32_t tile = t.order ? t.order[q] : q;
    const uint32_t ncyc = t.tile_cycles ? t.tile_cycles[tile] : s.uniform;
#define RT_SPACE make_space<V>(t.tpo, tile * t.tile_lanes, threadIdx.x, blockDim.x)
    for (uint32_t c = 0; c < ncyc; c++) {
      stim_items<V>(d, s, RT_SPACE, c);
      __syncthreads();
      for (uint32_t L = 0; L < d.n_layers; L++) {
        eval_layer<V, U>(d, s, L, RT_SPACE, c);
        __syncthreads();
      }
      commit_items<V>(d, s, RT_SPACE, c);
      __syncthreads();
      if (s.n_probe) {
        probe_items<V>(s, RT_SPACE, c);
        __syncthreads();
      }
    }
#undef RT_SPACE
  }
}

struct GridArgs {
  uint32_t* count;        // scratch: arrivals at the current barrier
  uint32_t* gen;          // scratch: barrier generation
  uint32_t expected;      // arrivals that complete a barrier (= gridDim.x)
  uint64_t timeout_ns;    // bounded wait per barrier
  uint32_t ncyc;
  FastDiv tpo;            // n_pad / V
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Software grid barrier (sense by generation counter).  Every wait is bounded:
// after timeout_ns the block sets *err and returns false; blocks that see *err
// leave at their next barrier, so the kernel always ends.
__device__ __forceinline__ bool grid_sync(const GridArgs& g, uint32_t* err, int* sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const uint32_t my = ld_acquire(g.gen);
    __threadfence();
    if (atomicAdd(g.count, 1u) == g.expected - 1u) {
      atomicExch(g.count, 0u);
      __threadfence();
      atomicAdd(g.gen, 1u);
    } else {
      const uint64_t t0 = globaltimer();
      while (ld_acquire(g.gen) == my) {
        if (ld_acquire(err) != 0u) { ok = 0; break; }
        if (globaltimer() - t0 > g.timeout_ns) { atomicOr(err, 1u); ok = 0; break; }
        __nanosleep(100);
      }
    }
    if (ld_acquire(err) != 0u) ok = 0;
    __threadfence();
    *sh_ok = ok;
  }
  __syncthreads();
  return *sh_ok != 0;
}

template <int V, int U, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_grid(DDesign d, DSim s, GridArgs g) {
  __shared__ int sh_ok;
  // the work mapping is recomputed per phase (a few integer ops) instead of
  // being held in registers across every barrier
#define RT_SPACE make_space<V>(g.tpo, 0u, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x)
  for (uint32_t c = 0; c < g.ncyc; c++) {
    stim_items<V>(d, s, RT_SPACE, c);
    if (!grid_sync(g, s.err, &sh_ok)) return;
    for (uint32_t L = 0; L < d.n_layers; L++) {
      eval_layer<V, U>(d, s, L, RT_SPACE, c);
      if (!grid_sync(g, s.err, &sh_ok)) return;
    }
    commit_items<V>(d, s, RT_SPACE, c);
    if (!grid_sync(g, s.err, &sh_ok)) return;
    if (s.n_probe) {
      probe_items<V>(s, RT_SPACE, c);
      if (!grid_sync(g, s.err, &sh_ok)) return;
    }
  }
#undef RT_SPACE
}

// GRID form with activity-aware evaluation (ops whose operands did not change
// in a 128-lane chunk are skipped there); counts evaluated / skipped items.
template <int V, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_grid_act(DDesign d, DSim s, GridArgs g) {
  __shared__ int sh_ok;
  uint32_t n_eval = 0, n_skip = 0;
#define RT_SPACE make_space<V>(g.tpo, 0u, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x)
  for (uint32_t c = 0; c < g.ncyc; c++) {
    stim_items<V>(d, s, RT_SPACE, c);
    if (!grid_sync(g, s.err, &sh_ok)) return;
    for (uint32_t L = 0; L < d.n_layers; L++) {
      eval_layer_act<V>(d, s, L, RT_SPACE, c, n_eval, n_skip);
      if (!grid_sync(g, s.err, &sh_ok)) return;
    }
    commit_items<V>(d, s, RT_SPACE, c);
    if (!grid_sync(g, s.err, &sh_ok)) return;
    if (s.n_probe) {
      probe_items<V>(s, RT_SPACE, c);
      if (!grid_sync(g, s.err, &sh_ok)) return;
    }
  }
#undef RT_SPACE
  for (int o = 16; o > 0; o >>= 1) {
    n_eval += __shfl_xor_sync(0xFFFFFFFFu, n_eval, o);
    n_skip += __shfl_xor_sync(0xFFFFFFFFu, n_skip, o);
  }
  if ((threadIdx.x & 31u) == 0 && (n_eval | n_skip)) {
    atomicAdd(&s.act_count[0], (unsigned long long)n_eval);
    atomicAdd(&s.act_count[1], (unsigned long long)n_skip);
  }
}


// Compiled variants of the persistent kernels: lanes per thread V, items in
// flight per thread U, launch bounds (MAXT threads per CTA, MINB CTAs per SM).
struct Variant {
  int V, U, maxt, minb;
  const void* tile;
  const void* grid;
};
struct VariantTable {
  const Variant* v;
  size_t n;
};
struct ActVariant {
  int V, maxt, minb;
  const void* grid;
};
struct ActVariantTable {
  const ActVariant* v;
  size_t n;
};
#define RT_VARIANT(V, U, T, B) {V, U, T, B, (const void*)k_tile<V, U, T, B>, (const void*)k_grid<V, U, T, B>}
#define RT_ACT_VARIANT(V, T, B) {V, T, B, (const void*)k_grid_act<V, T, B>}

VariantTable variants_v8();     // variants_v8.cu
VariantTable variants_v4();     // variants_v4.cu
VariantTable variants_v2_v1();  // variants_v2_v1.cu
ActVariantTable act_variants(); // variants_act.cu

}  // namespace rteaal
