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

// Barrier between two phases of a tile.  The phase's own staging copies (the
// next layer's descriptors, issued when the phase began) are complete in the
// issuing threads first; the cluster barrier then orders every thread's
// writes -- rows, staged descriptors -- before the next phase's reads, inside
// the CTA as across the cluster.
__device__ __forceinline__ void cluster_phase_sync() {
  cp_async_wait_all();
  cluster_arrive();
  cluster_wait();
}

// The per-layer row offsets (layer_off, layer_wide, layer_ext) in shared
// memory, loaded once per launch: [0, L] offsets, then [L] wide, then [L] ext.
__device__ __forceinline__ void load_layer_table(const DDesign& d, uint32_t* tab) {
  const uint32_t nl = d.n_layers;
  for (uint32_t i = threadIdx.x; i <= nl; i += blockDim.x) tab[i] = __ldg(&d.layer_off[i]);
  for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x) {
    tab[nl + 1 + i] = __ldg(&d.layer_wide[i]);
    tab[2 * nl + 1 + i] = __ldg(&d.layer_ext[i]);
  }
}

// Issue the copies of layer L's descriptors for this CTA into one of the two
// staging buffers (every thread takes a share); 0 rows if they do not fit.
__device__ __forceinline__ void stage_layer_tab(const DDesign& d, const uint32_t* tab, uint32_t L, const Stage& st,
                                                uint32_t cap, uint4* meta, uint32_t* dst) {
  if (L >= d.n_layers) return;
  const uint32_t o0 = tab[L], n = tab[L + 1] - o0;
  const uint32_t total = stage_rows(st, n);
  if (total > cap) return;
  for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const uint32_t i = idx / st.span, j = idx - i * st.span;
    const uint32_t r = st.R0 + i * st.per + j;
    if (r < n) {
      cp_async16(&meta[idx], &d.meta[o0 + r]);
      cp_async4(&dst[idx], &d.dst[o0 + r]);
    }
  }
}

template <int V, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_cluster(DDesign d, DSim s, ClusterArgs ca) {
  // dynamic shared memory: two staging buffers of stage_cap descriptors and
  // output rows, then the layer table
  extern __shared__ __align__(16) uint4 sm_stage[];
  uint4* meta[2] = {sm_stage, sm_stage + ca.stage_cap};
  uint32_t* dst0 = reinterpret_cast<uint32_t*>(sm_stage + 2 * ca.stage_cap);
  uint32_t* dst[2] = {dst0, dst0 + ca.stage_cap};
  uint32_t* tab = dst0 + 2 * ca.stage_cap;
  const uint32_t rank = cluster_rank(), nthreads = cluster_size() * blockDim.x;
  const uint32_t ct = rank * blockDim.x + threadIdx.x;
  const Stage st = stage_of_cluster_cta(ca.tpo, rank, nthreads);
  load_layer_table(d, tab);
  __syncthreads();
  for (uint32_t tile = cluster_id(); tile < ca.n_tiles; tile += cluster_count()) {
    const uint32_t ncyc = ca.tile_cycles ? ca.tile_cycles[tile] : s.uniform;
    const uint32_t base = tile * ca.tile_lanes;
#define RT_SPACE make_space<V>(ca.tpo, base, ct, nthreads)
    for (uint32_t c = 0; c < ncyc; c++) {
      if (ca.stage_cap) stage_layer_tab(d, tab, 0u, st, ca.stage_cap, meta[0], dst[0]);
      stim_items<V>(d, s, RT_SPACE, c);
      cluster_phase_sync();
      for (uint32_t L = 0; L < d.n_layers; L++) {
        const uint32_t b = L & 1u;
        if (ca.stage_cap) stage_layer_tab(d, tab, L + 1u, st, ca.stage_cap, meta[b ^ 1u], dst[b ^ 1u]);
        const uint32_t o0 = tab[L], n = tab[L + 1] - o0;
        const uint32_t total = stage_rows(st, n);
        const ItemSpace is = RT_SPACE;
        if (ca.stage_cap && is.row_stride && total && total <= ca.stage_cap) {
          if (is.row0 != NO_ROW && is.row0 < n) {
            const uint32_t am = act_mask<V>(s, is.lane, c);
            if (am) {
              const uint32_t nw = tab[d.n_layers + 1 + L] - o0, ne = tab[2 * d.n_layers + 1 + L] - o0;
              const uint32_t j = is.row0 - st.R0;
              uint32_t i = 0, r = is.row0;
              walk_staged<V, ROW_NARROW, 1>(d, s, i, r, nw, st, j, is.lane, am, meta[b], dst[b]);
              walk_staged<V, ROW_WIDE, 1>(d, s, i, r, ne, st, j, is.lane, am, meta[b], dst[b]);
              walk_staged<V, ROW_EXT, 1>(d, s, i, r, n, st, j, is.lane, am, meta[b], dst[b]);
            }
          }
        } else {
          eval_layer<V, 1>(d, s, L, is, c);
        }
        cluster_phase_sync();
      }
      commit_items<V>(d, s, RT_SPACE, c);
      cluster_phase_sync();
      if (s.n_probe) {
        probe_items<V>(s, RT_SPACE, c);
        cluster_phase_sync();
      }
    }
#undef RT_SPACE
  }
}

// ---- resident variant (few lanes): the whole compact state lives in the
// cluster's distributed shared memory.  The state's bytes (lane_bytes x lanes)
// are split into cluster-size slices of S bytes; CTA q keeps bytes
// [q S, (q + 1) S) in its shared memory, loaded from global memory when the
// launch starts and written back when it ends.  S is a multiple of 16 and
// every element is naturally aligned at its size, so an element never straddles
// two slices: it is one load or store at a generic address inside the
// cluster's shared-memory window (mapa).  Memories, stimulus states and probes
// stay in global memory.  One lane per thread; the cluster barrier orders the
// shared::cluster accesses of one phase before the next.
struct ResidentArgs {
  uint32_t ncyc;       // cycles of this step (lanes stop at their own budgets)
  uint32_t bytes;      // state bytes (lane_bytes x lanes)
  FastDiv slice;       // S
  FastDiv tpo;         // lanes (one lane per thread)
  uint32_t stage_cap;  // descriptors a CTA can stage (0: none)
};

__device__ __forceinline__ uint8_t* dsmem_map(uint8_t* p, uint32_t rank) {
  uint64_t r;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
  return reinterpret_cast<uint8_t*>(r);
}

// Element (row ref, lane) of the resident state.
__device__ __forceinline__ uint8_t* res_elem(uint8_t* const* base, const ResidentArgs& ra, uint32_t ref,
                                             uint32_t lane) {
  const uint32_t o = (ref & REF_OFF_MASK) * ra.tpo.d + (lane << (ref >> 30));
  const uint32_t q = fdiv(ra.slice, o);
  return base[q] + (o - q * ra.slice.d);
}

__device__ __forceinline__ uint64_t res_ld(uint8_t* const* base, const ResidentArgs& ra, uint32_t ref,
                                           uint32_t lane) {
  const uint8_t* p = res_elem(base, ra, ref, lane);
  switch (ref >> 30) {
    case 0: return *p;
    case 1: return *reinterpret_cast<const uint16_t*>(p);
    case 2: return *reinterpret_cast<const uint32_t*>(p);
    default: return *reinterpret_cast<const uint64_t*>(p);
  }
}

__device__ __forceinline__ void res_st(uint8_t* const* base, const ResidentArgs& ra, uint32_t ref, uint32_t lane,
                                       uint64_t v) {
  uint8_t* p = res_elem(base, ra, ref, lane);
  switch (ref >> 30) {
    case 0: *p = (uint8_t)v; break;
    case 1: *reinterpret_cast<uint16_t*>(p) = (uint16_t)v; break;
    case 2: *reinterpret_cast<uint32_t*>(p) = (uint32_t)v; break;
    default: *reinterpret_cast<uint64_t*>(p) = v; break;
  }
}

// (a2) one op for one lane from the resident state.
__device__ __forceinline__ void res_item(const DDesign& d, const DSim& s, uint8_t* const* base,
                                         const ResidentArgs& ra, const uint4& m, uint32_t dref, uint32_t lane) {
  uint64_t r;
  if (m.w & CTL_EXT) {
    const Lanes<1> x = ext_eval<1, Lanes<1>>(d.ext + m.x, m.w & 31u, m.y, [&](uint32_t ref) {
      Lanes<1> y;
      y.x[0] = res_ld(base, ra, ref, lane);
      return y;
    });
    r = x.x[0] & wmask(ctl_width(m.w));
  } else {
    const uint32_t ar = (m.w >> 5) & 3u;
    const uint64_t a = res_ld(base, ra, m.x, lane);
    const uint64_t b = ar >= 2 ? res_ld(base, ra, m.y, lane) : 0ull;
    const uint64_t c = ar >= 3 ? res_ld(base, ra, m.z, lane) : 0ull;
    r = (m.w & 31u) == OP_MEMRD ? eval_memrd(d, s, m.w, a, lane) : alu(m.w, a, b, c);
  }
  res_st(base, ra, dref, lane, r);
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_cluster_res(DDesign d, DSim s, ResidentArgs ra) {
  // dynamic shared memory: [S] state slice, two staging buffers, the layer table
  extern __shared__ __align__(16) uint8_t sm_res[];
  __shared__ uint8_t* base[16];
  const uint32_t S = ra.slice.d;
  uint8_t* slice = sm_res;
  uint4* meta[2] = {reinterpret_cast<uint4*>(sm_res + S), reinterpret_cast<uint4*>(sm_res + S) + ra.stage_cap};
  uint32_t* dst0 = reinterpret_cast<uint32_t*>(meta[1] + ra.stage_cap);
  uint32_t* dst[2] = {dst0, dst0 + ra.stage_cap};
  uint32_t* tab = dst0 + 2 * ra.stage_cap;
  const uint32_t rank = cluster_rank(), cs = cluster_size(), nthreads = cs * blockDim.x;
  const uint32_t ct = rank * blockDim.x + threadIdx.x;
  if (threadIdx.x < cs) base[threadIdx.x] = dsmem_map(slice, threadIdx.x);
  {  // this CTA's slice of the state from global memory
    const uint32_t lo = rank * S, hi = min(lo + S, ra.bytes);
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) slice[i - lo] = s.state[i];
  }
  load_layer_table(d, tab);
  const Stage st = stage_of_cluster_cta(ra.tpo, rank, nthreads);
  __syncthreads();
  cluster_arrive();
  cluster_wait();
#define RT_SPACE make_space<1>(ra.tpo, 0u, ct, nthreads)
  for (uint32_t c = 0; c < ra.ncyc; c++) {
    if (ra.stage_cap) stage_layer_tab(d, tab, 0u, st, ra.stage_cap, meta[0], dst[0]);
    // (a1) inputs
    if (s.stim_mode)
      for_rows<1>(RT_SPACE, d.n_inputs, [&](uint32_t j, uint32_t lane) {
        if (!lane_active(s, lane, c)) return;
        uint64_t x;
        if (s.stim_mode == 1) {
          x = s.xs[(size_t)j * s.n_pad + lane];
          x ^= x << 13;
          x ^= x >> 7;
          x ^= x << 17;
          s.xs[(size_t)j * s.n_pad + lane] = x;
        } else {
          x = __ldg(&s.stim[((size_t)c * d.n_inputs + j) * s.n_user + user_of(s, lane)]);
        }
        res_st(base, ra, __ldg(&d.in_ref[j]), lane, x & wmask(__ldg(&d.in_w[j])));
      });
    cluster_phase_sync();
    // (a2) layers
    for (uint32_t L = 0; L < d.n_layers; L++) {
      const uint32_t b = L & 1u;
      if (ra.stage_cap) stage_layer_tab(d, tab, L + 1u, st, ra.stage_cap, meta[b ^ 1u], dst[b ^ 1u]);
      const ItemSpace is = RT_SPACE;
      const uint32_t o0 = tab[L], n = tab[L + 1] - o0;
      const uint32_t total = stage_rows(st, n);
      if (is.row_stride && is.row0 != NO_ROW && lane_active(s, is.lane, c)) {
        const bool staged = ra.stage_cap && total && total <= ra.stage_cap;
        const uint32_t j = is.row0 - st.R0;
        uint32_t i = 0;
        for (uint32_t r = is.row0; r < n; r += is.row_stride, i++) {
          uint4 m;
          uint32_t dref;
          if (staged) {
            m = meta[b][i * st.span + j];
            dref = dst[b][i * st.span + j];
          } else {
            m = __ldg(&d.meta[o0 + r]);
            dref = __ldg(&d.dst[o0 + r]);
          }
          res_item(d, s, base, ra, m, dref, is.lane);
        }
      } else if (!is.row_stride) {  // more lanes than threads
        for_rows<1>(is, n, [&](uint32_t r, uint32_t lane) {
          if (lane_active(s, lane, c)) res_item(d, s, base, ra, __ldg(&d.meta[o0 + r]), __ldg(&d.dst[o0 + r]), lane);
        });
      }
      cluster_phase_sync();
    }
    // (a5) clock edge: registers, then memory write ports
    for_rows<1>(RT_SPACE, d.n_regs + d.n_mems, [&](uint32_t r, uint32_t lane) {
      if (!lane_active(s, lane, c)) return;
      if (r < d.n_regs) {
        const uint64_t mk = wmask(__ldg(&d.reg_w[r]));
        uint64_t v = res_ld(base, ra, __ldg(&d.reg_src[r]), lane) & mk;
        if (s.reset || (s.reset_lane && c < __ldg(&s.reset_lane[lane]))) v = __ldg(&d.reg_init[r]) & mk;
        res_st(base, ra, __ldg(&d.reg_ref[r]), lane, v);
      } else {
        const uint32_t mi = r - d.n_regs;
        const uint4 info = __ldg(&d.mem_info[mi]);
        const uint32_t p1 = __ldg(&d.mem_info[mi + 1]).w;
        const uint64_t mk = wmask(info.z);
        for (uint32_t p = info.w; p < p1; p++) {
          const uint4 w = __ldg(&d.wport[p]);
          if (res_ld(base, ra, w.y, lane) & 1ull) {
            const uint64_t a = res_ld(base, ra, w.z, lane) & (uint64_t)info.y;
            s.mem[((size_t)info.x + a) * s.n_pad + lane] = res_ld(base, ra, w.w, lane) & mk;
          }
        }
      }
    });
    cluster_phase_sync();
    // (a7) probes
    if (s.n_probe) {
      for_rows<1>(RT_SPACE, s.n_probe, [&](uint32_t p, uint32_t lane) {
        if (!lane_active(s, lane, c)) return;
        const uint64_t v = res_ld(base, ra, __ldg(&s.probe_slot[p]), lane);
        if (s.probe_changes) {
          uint64_t* prev = s.probe_prev + (size_t)p * s.n_pad + lane;
          if (*prev != v) {
            *prev = v;
            const unsigned long long k = atomicAdd(s.change_count, 1ull);
            if (k < s.change_cap) {
              uint64_t* rec = s.probe_out + 3 * k;
              rec[0] = (uint64_t)c | ((uint64_t)p << 32);
              rec[1] = (uint64_t)user_of(s, lane);
              rec[2] = v;
            }
          }
        } else {
          s.probe_out[((size_t)c * s.n_probe + p) * s.n_user + user_of(s, lane)] = v;
        }
      });
      cluster_phase_sync();
    }
  }
#undef RT_SPACE
  {  // the slice back to global memory
    const uint32_t lo = rank * S, hi = min(lo + S, ra.bytes);
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s.state[i] = slice[i - lo];
  }
  // no CTA may leave while another still reads its shared memory
  cluster_arrive();
  cluster_wait();
}

// Compiled variants: lanes per thread V, threads per CTA (one CTA per SM),
// state in global memory or resident in the cluster's shared memory.
struct ClusterVariant {
  int V, maxt;
  const void* fn;
  bool resident;
};
struct ClusterVariantTable {
  const ClusterVariant* v;
  size_t n;
};
#define RT_CLUSTER_VARIANT(V, T) {V, T, (const void*)k_cluster<V, T>, false}
#define RT_CLUSTER_RES_VARIANT(T) {1, T, (const void*)k_cluster_res<T>, true}
ClusterVariantTable variants_cluster();  // variants_cluster.cu

}  // namespace rteaal
