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
  unsigned long long* count;  // scratch (zeroed before the launch): arrivals at every barrier so far
  uint32_t expected;      // arrivals that complete a barrier (= gridDim.x)
  uint64_t timeout_ns;    // bounded wait per barrier
  uint32_t ncyc;
  FastDiv tpo;            // lane span / V
  uint32_t stage_cap;     // descriptors a CTA can stage in shared memory (0: none)
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Software grid barrier on one arrival count that only grows: barrier k of a
// launch is complete once the count reaches (k + 1) * expected, so a block's
// arrival is one atomic add, the last block to arrive has nothing to reset and
// no generation word is written.  The block's writes are ordered before its
// arrival by __syncthreads and a fence (release); the fence after the wait
// orders the next phase's reads after every block's arrival (acquire).  Every
// wait is bounded: after timeout_ns the block sets *err and returns false;
// blocks that see *err leave at their next barrier, so the kernel always ends.
// Called by one thread of the block; returns whether the block goes on.
__device__ __forceinline__ int grid_arrive_wait(const GridArgs& g, uint32_t* err) {
  __threadfence();
  uint32_t e = ld_relaxed(err);
  const unsigned long long old = atomicAdd(g.count, 1ull);
  const unsigned long long target = (old / g.expected + 1ull) * g.expected;
  if (old + 1ull < target) {
    const uint64_t t0 = globaltimer();
    for (;;) {
      const unsigned long long c = ld_relaxed64(g.count);
      e = ld_relaxed(err);
      if (c >= target || e != 0u) break;
      if (globaltimer() - t0 > g.timeout_ns) {
        atomicOr(err, 1u);
        e = 1u;
        break;
      }
      __nanosleep(32);
    }
  }
  __threadfence();
  return e == 0u;
}

__device__ __forceinline__ bool grid_sync(const GridArgs& g, uint32_t* err, int* sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) *sh_ok = grid_arrive_wait(g, err);
  __syncthreads();
  return *sh_ok != 0;
}
// ---- op descriptors staged in shared memory (the OIM of one layer for the
// rows this CTA evaluates), copied with cp.async while the CTA waits at the
// grid barrier before the layer, so that an item reads its descriptor from
// shared memory instead of carrying a global load in its chain.
//
// In the fixed mapping thread t keeps lane chunk t mod tpo and walks rows
// row0 = t / tpo, row0 + per, row0 + 2 per, ... (per = threads / tpo).  The
// CTA's threads have row0 in [R0, R0 + span), so at step i they need the
// contiguous rows [R0 + i per, R0 + i per + span): entry i * span + (row0 - R0).
struct Stage {
  uint32_t R0, span, per;  // span = 0: the CTA stages nothing (no rows, generic mapping)
};

__device__ __forceinline__ Stage stage_of_cta(const FastDiv& tpo) {
  Stage st{0, 0, 0};
  const uint32_t nthreads = gridDim.x * blockDim.x;
  if (nthreads < tpo.d) return st;  // generic mapping
  const uint32_t per = fdiv(tpo, nthreads), valid = per * tpo.d;
  const uint32_t t0 = blockIdx.x * blockDim.x;
  if (t0 >= valid) return st;
  const uint32_t t1 = min(t0 + blockDim.x, valid) - 1u;
  st.R0 = fdiv(tpo, t0);
  st.span = fdiv(tpo, t1) - st.R0 + 1u;
  st.per = per;
  return st;
}

// Descriptors the CTA needs for a layer of n rows (0 if it has none).
__device__ __forceinline__ uint32_t stage_rows(const Stage& st, uint32_t n) {
  if (!st.span || n <= st.R0) return 0;
  return (n - st.R0 + st.per - 1u) / st.per * st.span;
}

__device__ __forceinline__ void cp_async16(void* sm, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sm)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* sm, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(sm)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Issue the copies of layer L's descriptors for this CTA (every thread takes a share).
__device__ __forceinline__ void stage_layer(const DDesign& d, uint32_t L, const Stage& st, uint32_t cap,
                                            uint4* sm_meta, uint32_t* sm_dst) {
  const uint32_t o0 = __ldg(&d.layer_off[L]), n = __ldg(&d.layer_off[L + 1]) - o0;
  const uint32_t total = stage_rows(st, n);
  if (total > cap) return;  // does not fit: the layer reads its descriptors from global memory
  for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const uint32_t i = idx / st.span, j = idx - i * st.span;
    const uint32_t r = st.R0 + i * st.per + j;
    if (r < n) {
      cp_async16(&sm_meta[idx], &d.meta[o0 + r]);
      cp_async4(&sm_dst[idx], &d.dst[o0 + r]);
    }
  }
}

// Grid barrier that stages the next phase's descriptors while it waits: the
// copies start once every thread of the CTA is done with the current ones.
template <typename F>
__device__ __forceinline__ bool grid_sync_staging(const GridArgs& g, uint32_t* err, int* sh_ok, F&& stage) {
  __syncthreads();
  stage();
  if (threadIdx.x == 0) *sh_ok = grid_arrive_wait(g, err);
  cp_async_wait_all();
  __syncthreads();
  return *sh_ok != 0;
}

// This thread's rows of one kind with descriptors from shared memory (entry
// i * span + j of row row0 + i * per); advances (i, row) past the kind.
// Narrow rows go two at a time when U >= 2: both rows' operand loads are
// issued before either result is computed (two gathers in flight per thread;
// 32-bit lanes keep the pair within the registers a wide row needs alone).
template <int V, int KIND, int U>
__device__ __forceinline__ void walk_staged(const DDesign& d, const DSim& s, uint32_t& i, uint32_t& r,
                                            uint32_t r_end, const Stage& st, uint32_t j, uint32_t lane,
                                            uint32_t am, const uint4* sm_meta, const uint32_t* sm_dst) {
  if constexpr (KIND == ROW_NARROW && U >= 2) {
    const size_t np = s.n_pad;
    for (; r + st.per < r_end; r += 2u * st.per, i += 2u) {
      const uint32_t i0 = i * st.span + j, i1 = i0 + st.span;
      const uint4 m0 = sm_meta[i0], m1 = sm_meta[i1];
      const uint32_t ar0 = (m0.w >> 5) & 3u, ar1 = (m1.w >> 5) & 3u;
      Lanes32<V> a0, b0, c0, a1, b1, c1;
#pragma unroll
      for (int v = 0; v < V; v++) b0.x[v] = c0.x[v] = b1.x[v] = c1.x[v] = 0u;
      a0 = ldr32<V>(s.state, m0.x, np, lane);
      a1 = ldr32<V>(s.state, m1.x, np, lane);
      if (ar0 >= 2) b0 = ldr32<V>(s.state, m0.y, np, lane);
      if (ar1 >= 2) b1 = ldr32<V>(s.state, m1.y, np, lane);
      if (ar0 >= 3) c0 = ldr32<V>(s.state, m0.z, np, lane);
      if (ar1 >= 3) c1 = ldr32<V>(s.state, m1.z, np, lane);
      str32<V>(s.state, sm_dst[i0], np, lane, alu32_v<V>(m0.w, a0, b0, c0), am);
      str32<V>(s.state, sm_dst[i1], np, lane, alu32_v<V>(m1.w, a1, b1, c1), am);
    }
  }
  for (; r < r_end; r += st.per, i++) {
    const uint32_t idx = i * st.span + j;
    item_of_kind<V, KIND>(d, s, lane, sm_meta[idx], sm_dst[idx], am);
  }
}

// (a2) one layer with staged descriptors; falls back to eval_layer where the
// CTA could not stage them.  am: the thread's lane activity this cycle.
template <int V, int U>
__device__ __forceinline__ void eval_layer_staged(const DDesign& d, const DSim& s, uint32_t L, const ItemSpace& is,
                                                  uint32_t cyc, uint32_t am, const Stage& st, uint32_t cap,
                                                  const uint4* sm_meta, const uint32_t* sm_dst) {
  const uint32_t o0 = __ldg(&d.layer_off[L]), n = __ldg(&d.layer_off[L + 1]) - o0;
  const uint32_t total = stage_rows(st, n);
  if (!is.row_stride || total == 0 || total > cap) {  // rows in flight apply to staged narrow rows only
    eval_layer<V, 1>(d, s, L, is, cyc);
    return;
  }
  if (is.row0 == NO_ROW || is.row0 >= n || !am) return;
  const uint32_t nw = __ldg(&d.layer_wide[L]) - o0, ne = __ldg(&d.layer_ext[L]) - o0;
  const uint32_t j = is.row0 - st.R0;
  uint32_t i = 0, r = is.row0;
  walk_staged<V, ROW_NARROW, U>(d, s, i, r, nw, st, j, is.lane, am, sm_meta, sm_dst);
  walk_staged<V, ROW_WIDE, 1>(d, s, i, r, ne, st, j, is.lane, am, sm_meta, sm_dst);
  walk_staged<V, ROW_EXT, 1>(d, s, i, r, n, st, j, is.lane, am, sm_meta, sm_dst);
}

template <int V, int U, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_grid(DDesign d, DSim s, GridArgs g) {
  __shared__ int sh_ok;
  extern __shared__ __align__(16) uint4 sm_stage[];  // [stage_cap] descriptors, then [stage_cap] output rows
  uint4* sm_meta = sm_stage;
  uint32_t* sm_dst = reinterpret_cast<uint32_t*>(sm_stage + g.stage_cap);
  // the work mapping is recomputed per phase (a few integer ops) instead of
  // being held in registers across every barrier
#define RT_SPACE make_space<V>(g.tpo, 0u, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x)
#define RT_STAGE(L)                                                                            \
  [&] {                                                                                       \
    if (g.stage_cap && (L) < d.n_layers) stage_layer(d, (L), stage_of_cta(g.tpo), g.stage_cap, sm_meta, sm_dst); \
  }
  for (uint32_t c = 0; c < g.ncyc; c++) {
    stim_items<V>(d, s, RT_SPACE, c);
    uint32_t am = 0;  // the thread's lane activity this cycle (fixed mapping), loaded during the barrier
    {
      const ItemSpace is = RT_SPACE;
      if (is.row_stride && is.row0 != NO_ROW) am = act_mask<V>(s, is.lane, c);
    }
    if (!grid_sync_staging(g, s.err, &sh_ok, RT_STAGE(0u))) return;
    for (uint32_t L = 0; L < d.n_layers; L++) {
      if (g.stage_cap)
        eval_layer_staged<V, U>(d, s, L, RT_SPACE, c, am, stage_of_cta(g.tpo), g.stage_cap, sm_meta, sm_dst);
      else
        eval_layer<V, 1>(d, s, L, RT_SPACE, c);
      if (!grid_sync_staging(g, s.err, &sh_ok, RT_STAGE(L + 1u))) return;
    }
#undef RT_STAGE
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

// one translation unit per table (variants_<name>.cu), compiled in parallel
VariantTable variants_v8a();
VariantTable variants_v8b();
VariantTable variants_v8c();
VariantTable variants_v8d();
VariantTable variants_v4a();
VariantTable variants_v4b();
VariantTable variants_v4c();
VariantTable variants_v2();
VariantTable variants_v1();
ActVariantTable variants_act_a();
ActVariantTable variants_act_b();

}  // namespace rteaal
