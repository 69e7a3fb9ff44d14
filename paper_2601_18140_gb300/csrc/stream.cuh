// stream.cuh -- the streaming form: operand gathers through the bulk-copy (TMA)
// engine into a shared-memory ring, computation from shared memory.
//
// One CTA per SM walks every layer of every cycle over all lanes (grid barrier
// between layers, as in the grid form).  An item is one op for a chunk of
// CHUNK consecutive lanes.  CTA b owns a contiguous range of the layer's ops
// (all their chunks, op-major).  Per item:
//   producer (one thread): wait until the ring slot is free (empty barrier),
//     write the op's descriptor into the slot, announce the byte count on the
//     slot's full barrier and issue one cp.async.bulk per operand row segment
//     (CHUNK << class bytes, contiguous in the compact layout);
//   consumer warp (items round-robin over NCW warps): wait on the full
//     barrier, evaluate the CHUNK lanes from shared memory (4 packed lanes per
//     thread per step), store the results to global memory, release the slot.
// The ring keeps NS items of operand bytes in flight per SM without holding
// registers, which is what the gather needs: it is latency-bound, not
// instruction-bound, when every thread keeps one dependent load chain alive.
// Every mbarrier wait is bounded (%globaltimer); on a timeout the CTA records
// the error, drains its own copies in flight (bounded) and leaves at the next
// grid barrier.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace rteaal {

constexpr uint32_t STREAM_NS = 64;                     // item (descriptor) slots
constexpr uint32_t STREAM_CHUNK_MAX = 2048;            // lanes per item
constexpr uint32_t STREAM_RING = 160 * 1024;           // operand bytes in flight per SM
constexpr uint32_t STREAM_V = 4;                       // lanes per consumer thread per step
constexpr uint32_t STREAM_ACT_WORDS = 2048;            // activity bitmap: up to 65,536 lanes

struct StreamArgs {
  uint32_t chunk;       // lanes per item (divides n_pad, multiple of 32 * STREAM_V, <= STREAM_CHUNK_MAX)
  uint32_t n_chunks;    // n_pad / chunk
};

struct __align__(16) SlotInfo {
  uint4 meta;
  uint32_t dst, lane0;
  uint32_t off[3];               // ring byte offset of each operand segment
  uint32_t pad;
  unsigned long long start;      // monotonic ring position of the item's first byte
};

constexpr uint32_t stream_smem_bytes() {
  return STREAM_RING + STREAM_NS * (uint32_t)sizeof(SlotInfo) + 2 * STREAM_NS * 8 +
         STREAM_ACT_WORDS * 4 + 64;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t stream_clock() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase with the given parity; false after timeout_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = stream_clock();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (stream_clock() - t0 > timeout_ns) return false;
  }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Order this thread's later bulk-copy (async proxy) reads after the generic
// writes that the preceding barrier made visible.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// STREAM_V lanes of an operand segment in shared memory (class k, lane offset sub).
__device__ __forceinline__ Lanes<STREAM_V> lds4(const uint8_t* seg, uint32_t k, uint32_t sub) {
  Lanes<STREAM_V> r;
  const uint8_t* p = seg + (sub << k);
  switch (k) {
    case 0: {
      const uint32_t t = *reinterpret_cast<const uint32_t*>(p);
      r.x[0] = t & 0xFFu;
      r.x[1] = (t >> 8) & 0xFFu;
      r.x[2] = (t >> 16) & 0xFFu;
      r.x[3] = t >> 24;
    } break;
    case 1: {
      const uint2 t = *reinterpret_cast<const uint2*>(p);
      r.x[0] = t.x & 0xFFFFu;
      r.x[1] = t.x >> 16;
      r.x[2] = t.y & 0xFFFFu;
      r.x[3] = t.y >> 16;
    } break;
    case 2: {
      const uint4 t = *reinterpret_cast<const uint4*>(p);
      r.x[0] = t.x;
      r.x[1] = t.y;
      r.x[2] = t.z;
      r.x[3] = t.w;
    } break;
    default: {
      const ulonglong2 t0 = reinterpret_cast<const ulonglong2*>(p)[0];
      const ulonglong2 t1 = reinterpret_cast<const ulonglong2*>(p)[1];
      r.x[0] = t0.x;
      r.x[1] = t0.y;
      r.x[2] = t1.x;
      r.x[3] = t1.y;
    } break;
  }
  return r;
}

// Evaluate one item from its ring slot (one consumer warp).
__device__ __forceinline__ void stream_consume(const DDesign& d, const DSim& s, const SlotInfo& si,
                                               const uint8_t* ring, uint32_t chunk, uint32_t cyc,
                                               uint32_t lane_id, const uint32_t* act) {
  const uint4 m = si.meta;
  const uint32_t ctl = m.w;
  const size_t np = s.n_pad;
  const uint32_t ar = (ctl >> 5) & 3u;
  const uint32_t ka = m.x >> 30, kb = m.y >> 30, kc = m.z >> 30;
  const uint8_t* sa = ring + si.off[0];
  const uint8_t* sb = ring + si.off[1];
  const uint8_t* sc = ring + si.off[2];
  for (uint32_t sub = lane_id * STREAM_V; sub < chunk; sub += 32 * STREAM_V) {
    const uint32_t lane = si.lane0 + sub;
    const uint32_t am = act ? (act[lane >> 5] >> (lane & 31u)) & 0xFu : act_mask<STREAM_V>(s, lane, cyc);
    if (!am) continue;
    Lanes<STREAM_V> r;
    if (ctl & CTL_EXT) {
      r = eval_ext_v<STREAM_V>(d, s, m, lane);
    } else {
      Lanes<STREAM_V> a = lds4(sa, ka, sub), b, c;
#pragma unroll
      for (int v = 0; v < (int)STREAM_V; v++) b.x[v] = c.x[v] = 0;
      if (ar >= 2) b = lds4(sb, kb, sub);
      if (ar >= 3) c = lds4(sc, kc, sub);
      if ((ctl & 31u) == OP_MEMRD) {
#pragma unroll
        for (int v = 0; v < (int)STREAM_V; v++) r.x[v] = eval_memrd(d, s, ctl, a.x[v], lane + v);
      } else {
        r = alu_v<STREAM_V>(ctl, a, b, c);
      }
    }
    str<STREAM_V>(s.state, si.dst, np, lane, r, am);
  }
}

template <int NCW>
__global__ void __launch_bounds__(32 * (NCW + 1), 1) k_stream(DDesign d, DSim s, GridArgs g, StreamArgs sa) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* ring = smem;
  SlotInfo* info = reinterpret_cast<SlotInfo*>(smem + STREAM_RING);
  uint64_t* full = reinterpret_cast<uint64_t*>(info + STREAM_NS);
  uint64_t* empty = full + STREAM_NS;
  uint32_t* act_bits = reinterpret_cast<uint32_t*>(empty + STREAM_NS);
  // per-cycle lane activity in shared memory (one bit per lane) when it fits
  const uint32_t act_words = (s.n_pad + 31) / 32;
  const uint32_t* act = act_words <= STREAM_ACT_WORDS ? act_bits : nullptr;
  __shared__ int sh_ok;
  __shared__ int sh_bad_store;
  __shared__ uint32_t sh_issued_store;  // items whose copies the producer issued (monotonic)
  volatile int* sh_bad = &sh_bad_store;
  volatile uint32_t* sh_issued = &sh_issued_store;
  const uint32_t warp = threadIdx.x / 32, lane_id = threadIdx.x % 32;
  const bool producer = warp == (uint32_t)NCW;
  if (threadIdx.x == 0) {
    for (uint32_t i = 0; i < STREAM_NS; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sh_bad = 0;
    *sh_issued = 0;
  }
  __syncthreads();
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x, nthreads = gridDim.x * blockDim.x;
  uint32_t kk = 0;      // items this CTA has passed through its ring (all warps agree)
  unsigned long long pos = 0;  // producer: next free monotonic ring byte
  uint32_t oldest = 0;         // producer: oldest item whose slot / bytes are not yet known free
#define RT_SPACE make_space<STREAM_V>(g.tpo, 0u, gtid, nthreads)
  for (uint32_t c = 0; c < g.ncyc; c++) {
    if (act)
      for (uint32_t w = threadIdx.x; w < act_words; w += blockDim.x) {
        uint32_t bits = 0;
        for (uint32_t b = 0; b < 32; b++)
          if (lane_active(s, w * 32 + b, c)) bits |= 1u << b;
        act_bits[w] = bits;
      }
    stim_items<STREAM_V>(d, s, RT_SPACE, c);
    if (!grid_sync(g, s.err, &sh_ok)) return;
    for (uint32_t L = 0; L < d.n_layers; L++) {
      const uint32_t o0 = __ldg(&d.layer_off[L]), o1 = __ldg(&d.layer_off[L + 1]);
      const uint32_t n_ops = o1 - o0;
      const uint32_t r0 = (uint32_t)((uint64_t)n_ops * blockIdx.x / gridDim.x);
      const uint32_t r1 = (uint32_t)((uint64_t)n_ops * (blockIdx.x + 1) / gridDim.x);
      const uint32_t n_items = (r1 - r0) * sa.n_chunks;
      if (producer) {
        // one issuing lane; monotonic byte positions: the ring segment of item k
        // is [start, end); space is reclaimed from the oldest item still in use
        if (lane_id == 0) {
          fence_proxy_async();
          for (uint32_t j = 0; j < n_items; j++) {
            if (*sh_bad) break;
            const uint32_t k = kk + j, slot = k % STREAM_NS, par = (k / STREAM_NS) & 1u;
            const uint32_t jr = j / sa.n_chunks;
            const uint32_t op = o0 + r0 + jr;
            const uint32_t lane0 = (j - jr * sa.n_chunks) * sa.chunk;
            const uint4 m = __ldg(&d.meta[op]);
            const uint32_t ar = (m.w & CTL_EXT) ? 0u : (m.w >> 5) & 3u;
            const uint32_t refs[3] = {m.x, m.y, m.z};
            uint32_t need = 0;
            for (uint32_t o = 0; o < ar; o++) need += sa.chunk << (refs[o] >> 30);
            // contiguous placement: skip to the next ring lap if the item would wrap
            unsigned long long p0 = pos;
            if ((p0 % STREAM_RING) + need > STREAM_RING) p0 = (p0 / STREAM_RING + 1) * STREAM_RING;
            bool ok = true;
            // free the descriptor slot (item k - NS) and the ring bytes up to p0 + need by
            // waiting for the oldest items' release (item counters compared by difference)
            while (ok && (k - oldest >= STREAM_NS ||
                          (k != oldest && p0 + need > info[oldest % STREAM_NS].start + STREAM_RING))) {
              ok = mbar_wait(&empty[oldest % STREAM_NS], (oldest / STREAM_NS) & 1u, g.timeout_ns);
              oldest++;
            }
            if (!ok) {
              atomicOr(s.err, 2u);
              *sh_bad = 1;
              break;
            }
            SlotInfo& si = info[slot];
            si.meta = m;
            si.dst = __ldg(&d.dst[op]);
            si.lane0 = lane0;
            si.start = p0;
            unsigned long long q = p0;
            for (uint32_t o = 0; o < 3; o++) {
              si.off[o] = (uint32_t)(q % STREAM_RING);
              if (o < ar) q += sa.chunk << (refs[o] >> 30);
            }
            pos = q;
            if (ar == 0) {
              mbar_arrive(&full[slot]);  // operands read from global by the consumer
            } else {
              mbar_arrive_expect_tx(&full[slot], need);
              for (uint32_t o = 0; o < ar; o++)
                bulk_g2s(ring + si.off[o], elem(s.state, refs[o], s.n_pad, lane0), sa.chunk << (refs[o] >> 30),
                         &full[slot]);
            }
            *sh_issued = k + 1u;
            (void)par;
          }
        }
      } else {
        for (uint32_t j = warp; j < n_items; j += NCW) {
          const uint32_t k = kk + j, slot = k % STREAM_NS, par = (k / STREAM_NS) & 1u;
          int ok = 1;
          if (lane_id == 0) {
            ok = *sh_bad ? 0 : (mbar_wait(&full[slot], par, g.timeout_ns) ? 1 : 2);
            if (ok == 2) {
              atomicOr(s.err, 2u);
              *sh_bad = 1;
            }
          }
          ok = __shfl_sync(0xFFFFFFFFu, ok, 0);  // warp-uniform decision
          if (ok != 1) break;
          stream_consume(d, s, info[slot], ring, sa.chunk, c, lane_id, act);
          __syncwarp();
          if (lane_id == 0) mbar_arrive(&empty[slot]);
        }
      }
      kk += n_items;
      __syncthreads();
      if (*sh_bad) {
        // drain: wait (bounded) for the copies this CTA actually issued and that
        // may still be in flight (the last NS items up to the producer's count),
        // then leave; a drain wait that gives up is reported as its own bit
        __syncthreads();
        if (threadIdx.x == 0) {
          const uint32_t issued = *sh_issued;
          const uint32_t first = issued > STREAM_NS ? issued - STREAM_NS : 0;
          for (uint32_t k = first; k < issued; k++)
            if (!mbar_wait(&full[k % STREAM_NS], (k / STREAM_NS) & 1u, g.timeout_ns)) {
              atomicOr(s.err, 4u);
              break;
            }
        }
        __syncthreads();
        grid_sync(g, s.err, &sh_ok);
        return;
      }
      if (!grid_sync(g, s.err, &sh_ok)) return;
    }
    commit_items<STREAM_V>(d, s, RT_SPACE, c);
    if (!grid_sync(g, s.err, &sh_ok)) return;
    if (s.n_probe) {
      probe_items<STREAM_V>(s, RT_SPACE, c);
      if (!grid_sync(g, s.err, &sh_ok)) return;
    }
  }
#undef RT_SPACE
}

}  // namespace rteaal
