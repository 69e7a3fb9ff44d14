// cluster.cuh -- the cluster form: thread-block clusters (up to 16 CTAs on
// neighbouring SMs) each own a tile of lanes and walk every layer of every
// cycle of that tile, with the hardware cluster barrier between layers.
//
// Instances are independent, so the rows of a lane tile are read and written
// by its own cluster only: the LI_{i+1} <- LO_i step (a barrier, rows being
// global) needs the cluster's CTAs to agree, not the whole grid.  The
// barrier.cluster arrive (release) / wait (acquire) pair orders every CTA's
// row writes of one layer before the next layer's reads, at cluster scope,
// without the software grid barrier's atomics and spin (and without a bounded
// wait: the hardware schedules a cluster's CTAs together).  Cluster c takes
// tiles c, c + clusters, ...; each tile runs its own cycle count.  Inside a
// cluster the work mapping is the grid form's, over the cluster's threads and
// the tile's lanes, and each CTA stages the descriptors of the rows its
// threads evaluate in shared memory between arrive and wait.
#pragma once
#include <cstdint>

#include "kernels.cuh"
#include "persistent.cuh"

namespace rteaal {

struct ClusterArgs {
  uint32_t tile_lanes;            // lanes per tile (a multiple of V)
  uint32_t n_tiles;
  const uint32_t* tile_cycles;    // [n_tiles] cycles of each tile this step, or null (uniform)
  FastDiv tpo;                    // tile_lanes / V
  uint32_t stage_cap;             // descriptors a CTA can stage (0: none)
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Stage geometry of this CTA inside its cluster (the grid form's, over the
// cluster's threads): see Stage in persistent.cuh.
__device__ __forceinline__ Stage stage_of_cluster_cta(const FastDiv& tpo, uint32_t rank, uint32_t nthreads) {
  Stage st{0, 0, 0};
  if (nthreads < tpo.d) return st;
  const uint32_t per = fdiv(tpo, nthreads), valid = per * tpo.d;
  const uint32_t t0 = rank * blockDim.x;
  if (t0 >= valid) return st;
  const uint32_t t1 = min(t0 + blockDim.x, valid) - 1u;
  st.R0 = fdiv(tpo, t0);
  st.span = fdiv(tpo, t1) - st.R0 + 1u;
  st.per = per;
  return st;
}

// Barrier between two phases of a tile: the CTA's threads are done with the
// current descriptors, the next layer's are staged while the cluster waits.
template <typename F>
__device__ __forceinline__ void cluster_phase_sync(F&& stage) {
  __syncthreads();
  cluster_arrive();
  stage();
  cluster_wait();
  cp_async_wait_all();
  __syncthreads();
}

template <int V, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_cluster(DDesign d, DSim s, ClusterArgs ca) {
  extern __shared__ __align__(16) uint4 sm_stage[];  // [stage_cap] descriptors, then [stage_cap] output rows
  uint4* sm_meta = sm_stage;
  uint32_t* sm_dst = reinterpret_cast<uint32_t*>(sm_stage + ca.stage_cap);
  const uint32_t rank = cluster_rank(), nthreads = cluster_size() * blockDim.x;
  const uint32_t ct = rank * blockDim.x + threadIdx.x;
  const Stage st = stage_of_cluster_cta(ca.tpo, rank, nthreads);
  for (uint32_t tile = cluster_id(); tile < ca.n_tiles; tile += cluster_count()) {
    const uint32_t ncyc = ca.tile_cycles ? ca.tile_cycles[tile] : s.uniform;
    const uint32_t base = tile * ca.tile_lanes;
#define RT_SPACE make_space<V>(ca.tpo, base, ct, nthreads)
#define RT_STAGE(L)                                                                                  \
  [&] {                                                                                             \
    if (ca.stage_cap && (L) < d.n_layers) stage_layer(d, (L), st, ca.stage_cap, sm_meta, sm_dst);   \
  }
    for (uint32_t c = 0; c < ncyc; c++) {
      stim_items<V>(d, s, RT_SPACE, c);
      cluster_phase_sync(RT_STAGE(0u));
      for (uint32_t L = 0; L < d.n_layers; L++) {
        if (ca.stage_cap)
          eval_layer_staged<V, 1>(d, s, L, RT_SPACE, c, st, ca.stage_cap, sm_meta, sm_dst);
        else
          eval_layer<V, 1>(d, s, L, RT_SPACE, c);
        cluster_phase_sync(RT_STAGE(L + 1u));
      }
      commit_items<V>(d, s, RT_SPACE, c);
      cluster_phase_sync([] {});
      if (s.n_probe) {
        probe_items<V>(s, RT_SPACE, c);
        cluster_phase_sync([] {});
      }
    }
#undef RT_STAGE
#undef RT_SPACE
  }
}

// Compiled variants: lanes per thread V, threads per CTA (one CTA per SM).
struct ClusterVariant {
  int V, maxt;
  const void* fn;
};
struct ClusterVariantTable {
  const ClusterVariant* v;
  size_t n;
};
#define RT_CLUSTER_VARIANT(V, T) {V, T, (const void*)k_cluster<V, T>}
ClusterVariantTable variants_cluster();  // variants_cluster.cu

}  // namespace rteaal
