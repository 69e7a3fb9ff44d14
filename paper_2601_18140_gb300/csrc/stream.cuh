// stream.cuh -- the streaming form: every warp feeds its own shared-memory ring
// with bulk copies (TMA engine) of its items' operand row segments and
// evaluates them from shared memory.
//
// One CTA per SM walks every layer of every cycle over the live lanes (grid
// barrier between layers, as in the grid form).  An item is one op for a chunk
// of CH = 128 H consecutive lanes (H = 1 or 2); thread t of a warp owns lanes
// {4t .. 4t+3} of each 128-lane half of the chunk, so that its operand bytes
// are one conflict-free shared-memory access per half and its results one
// coalesced store per half.  Warp w keeps one chunk for the whole launch
// (w mod chunks) and walks the rows w / chunks, + W / chunks, ... of every
// layer (W warps in all).  Per item, lane 0
//   * reads the op's descriptor (staged in shared memory during the grid
//     barrier before the layer),
//   * reserves the operand bytes in the warp's ring (a FIFO of monotonic byte
//     positions), writes the item's slot record, announces the byte count on
//     the slot's mbarrier and issues one cp.async.bulk per operand segment
//     (CH << class bytes, contiguous in the compact layout);
// and the whole warp later waits on that mbarrier, evaluates the CH lanes from
// shared memory and stores the results to global memory.  Up to SLOTS items
// (at most RING bytes) are in flight per warp, with no registers held for
// them: the gather's latency is covered by the copy engine, and the threads
// only compute.  Ops with more than three operands read them from global
// memory instead (their slot carries no bytes).
//
// Every mbarrier wait is bounded (%globaltimer); on a timeout the warp records
// the error, waits (bounded) for the copies it issued and leaves at the next
// grid barrier with the rest of the grid.
#pragma once
#include <cstdint>

#include "kernels.cuh"
#include "persistent.cuh"

namespace rteaal {

constexpr uint32_t STREAM_WARPS = 16;     // warps per CTA (one CTA per SM)
constexpr uint32_t STREAM_RING = 8192;    // operand bytes per warp
constexpr uint32_t STREAM_SLOTS = 8;      // items in flight per warp
constexpr uint32_t STREAM_DESC = 128;     // descriptors staged per warp and layer
constexpr uint32_t STREAM_V = 4;          // lanes per thread in the stimulus / edge / probe phases
static_assert(3u * (256u << 3) <= STREAM_RING, "the largest item must fit the ring");

struct StreamArgs {
  uint32_t half;       // H: items of 128 H lanes
  uint32_t n_chunks;   // items per row over the lane span (span / (128 H))
};

struct __align__(16) SlotInfo {
  uint4 meta;
  uint32_t dst;
  uint32_t off[2];      // ring byte offsets of operands 0, 1 (operand 2 follows operand 1)
  uint32_t end;         // monotonic ring position just past the item's bytes
};

struct __align__(16) WarpArea {
  uint8_t ring[STREAM_RING];
  uint4 dmeta[STREAM_DESC];
  uint32_t ddst[STREAM_DESC];
  SlotInfo slot[STREAM_SLOTS];
  uint64_t full[STREAM_SLOTS];
};

constexpr uint32_t stream_smem_bytes() { return STREAM_WARPS * (uint32_t)sizeof(WarpArea); }

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

// Bounded wait for the phase with the given parity; false after timeout_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > timeout_ns) return false;
  }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Order the warp's earlier generic-proxy reads of a consumed item before later
// bulk copies (async proxy) into the same bytes.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 4 lanes of an operand segment in shared memory (class k <= 2), from lane
// offset sub (a multiple of 4): zero-extended to 32 bits.
__device__ __forceinline__ void lds32x4(const uint8_t* seg, uint32_t k, uint32_t sub, uint32_t* x) {
  const uint8_t* p = seg + (sub << k);
  if (k == 0) {
    const uint32_t t = *reinterpret_cast<const uint32_t*>(p);
#pragma unroll
    for (int v = 0; v < 4; v++) x[v] = __byte_perm(t, 0u, 0x4440u + v);
  } else if (k == 1) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    x[0] = t.x & 0xFFFFu; x[1] = t.x >> 16;
    x[2] = t.y & 0xFFFFu; x[3] = t.y >> 16;
  } else {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
  }
}

// The same for any class, zero-extended to 64 bits.
__device__ __forceinline__ Lanes<4> lds64x4(const uint8_t* seg, uint32_t k, uint32_t sub) {
  Lanes<4> r;
  if (k == 3) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(seg + (sub << 3));
    const ulonglong2 t0 = p[0], t1 = p[1];
    r.x[0] = t0.x; r.x[1] = t0.y; r.x[2] = t1.x; r.x[3] = t1.y;
  } else {
    uint32_t x[4];
    lds32x4(seg, k, sub, x);
#pragma unroll
    for (int v = 0; v < 4; v++) r.x[v] = x[v];
  }
  return r;
}

// Evaluate one item from its slot: thread lane_id owns lanes {4 lane_id ..
// + 3} of each 128-lane half of the chunk starting at lane0; am: bit 4h + v =
// lane 128 h + 4 lane_id + v active.
template <int H>
__device__ __forceinline__ void stream_item(const DDesign& d, const DSim& s, const SlotInfo& si,
                                            const uint8_t* ring, uint32_t lane0, uint32_t lane_id, uint32_t am) {
  const uint4 m = si.meta;
  const uint32_t ctl = m.w;
  const size_t np = s.n_pad;
  const uint32_t sub = 4u * lane_id;
  if (ctl & CTL_EXT) {  // operands from global memory
#pragma unroll
    for (int h = 0; h < H; h++) {
      const uint32_t lane = lane0 + 128u * h + sub, mk = (am >> (4 * h)) & 15u;
      if (!mk) continue;
      if (ctl & CTL_NARROW)
        str32<4>(s.state, si.dst, np, lane, eval_ext32_v<4>(d, s, m, lane), mk);
      else
        str<4>(s.state, si.dst, np, lane, eval_ext_v<4>(d, s, m, lane), mk);
    }
    return;
  }
  const uint32_t ar = (ctl >> 5) & 3u;
  const uint32_t ka = m.x >> 30, kb = m.y >> 30, kc = m.z >> 30;
  const uint32_t CH = 128u * H;
  const uint8_t* sa = ring + si.off[0];
  const uint8_t* sb = ring + si.off[1];
  const uint8_t* sc = sb + (CH << kb);
  if (ctl & CTL_NARROW) {
    Lanes32<4 * H> a, b, c;
#pragma unroll
    for (int h = 0; h < H; h++) {
      lds32x4(sa + ((128u * h) << ka), ka, sub, &a.x[4 * h]);
#pragma unroll
      for (int v = 0; v < 4; v++) b.x[4 * h + v] = c.x[4 * h + v] = 0u;
      if (ar >= 2) lds32x4(sb + ((128u * h) << kb), kb, sub, &b.x[4 * h]);
      if (ar >= 3) lds32x4(sc + ((128u * h) << kc), kc, sub, &c.x[4 * h]);
    }
    const Lanes32<4 * H> r = alu32_v<4 * H>(ctl, a, b, c);
#pragma unroll
    for (int h = 0; h < H; h++) {
      const uint32_t mk = (am >> (4 * h)) & 15u;
      if (!mk) continue;
      Lanes32<4> q;
#pragma unroll
      for (int v = 0; v < 4; v++) q.x[v] = r.x[4 * h + v];
      str32<4>(s.state, si.dst, np, lane0 + 128u * h + sub, q, mk);
    }
  } else {  // 64-bit lanes, one half at a time
#pragma unroll
    for (int h = 0; h < H; h++) {
      const uint32_t mk = (am >> (4 * h)) & 15u;
      if (!mk) continue;
      const uint32_t lane = lane0 + 128u * h + sub;
      const Lanes<4> a = lds64x4(sa + ((128u * h) << ka), ka, sub);
      Lanes<4> b, c;
#pragma unroll
      for (int v = 0; v < 4; v++) b.x[v] = c.x[v] = 0ull;
      if (ar >= 2) b = lds64x4(sb + ((128u * h) << kb), kb, sub);
      if (ar >= 3) c = lds64x4(sc + ((128u * h) << kc), kc, sub);
      str<4>(s.state, si.dst, np, lane, apply<4>(d, s, m, a, b, c, lane), mk);
    }
  }
}

// Warp w's place in the item space of a layer: its chunk (fixed for the
// launch), its first row and the stride between its rows (0: the warp has no
// rows -- the warps beyond a multiple of the chunk count).
struct WarpRows {
  uint32_t chunk, row0, stride;
};

__device__ __forceinline__ WarpRows warp_rows(uint32_t w, uint32_t n_warps, uint32_t n_chunks) {
  WarpRows wr;
  wr.stride = n_warps / n_chunks;
  wr.chunk = w % n_chunks;
  wr.row0 = w / n_chunks;
  if (wr.row0 >= wr.stride) wr.stride = 0;
  return wr;
}

// Stage the descriptors of the warp's rows of layer L (its first STREAM_DESC
// rows) into its area; every lane copies a share (cp.async, completed before
// the grid barrier ends).
__device__ __forceinline__ void stream_stage(const DDesign& d, uint32_t L, const WarpRows& wr, WarpArea* wa,
                                             uint32_t lane_id) {
  if (!wr.stride || L >= d.n_layers) return;
  const uint32_t o0 = __ldg(&d.layer_off[L]), n = __ldg(&d.layer_off[L + 1]) - o0;
  for (uint32_t i = lane_id; i < STREAM_DESC; i += 32u) {
    const uint32_t r = wr.row0 + i * wr.stride;
    if (r >= n) break;
    cp_async16(&wa->dmeta[i], &d.meta[o0 + r]);
    cp_async4(&wa->ddst[i], &d.dst[o0 + r]);
  }
}

template <int H>
__global__ void __launch_bounds__(32 * STREAM_WARPS, 1) k_stream(DDesign d, DSim s, GridArgs g, StreamArgs sa) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ int sh_ok;
  const uint32_t warp = threadIdx.x / 32u, lane_id = threadIdx.x % 32u;
  WarpArea* wa = reinterpret_cast<WarpArea*>(smem) + warp;
  if (lane_id == 0) {
    for (uint32_t i = 0; i < STREAM_SLOTS; i++) mbar_init(&wa->full[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint32_t n_warps = gridDim.x * STREAM_WARPS;
  const WarpRows wr = warp_rows(blockIdx.x * STREAM_WARPS + warp, n_warps, sa.n_chunks);
  const uint32_t CH = 128u * H, lane0 = wr.chunk * CH;
  uint32_t uses = 0;  // items that went through this warp's slots since launch (slot and parity)
  bool bad = false;
#define RT_SPACE make_space<STREAM_V>(g.tpo, 0u, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x)
  for (uint32_t c = 0; c < g.ncyc; c++) {
    // lane activity of this thread's lanes in the cycle (the warp's chunk is fixed)
    uint32_t am = 0;
    if (wr.stride)
#pragma unroll
      for (int h = 0; h < H; h++) am |= act_mask<4>(s, lane0 + 128u * h + 4u * lane_id, c) << (4 * h);
    const bool warp_live = __ballot_sync(0xFFFFFFFFu, am != 0u) != 0u;
    stim_items<STREAM_V>(d, s, RT_SPACE, c);
    if (!grid_sync_staging(g, s.err, &sh_ok, [&] { stream_stage(d, 0u, wr, wa, lane_id); })) return;
    for (uint32_t L = 0; L < d.n_layers; L++) {
      const uint32_t o0 = __ldg(&d.layer_off[L]), n = __ldg(&d.layer_off[L + 1]) - o0;
      const uint32_t ni = (wr.stride && warp_live && wr.row0 < n) ? (n - wr.row0 + wr.stride - 1u) / wr.stride : 0u;
      uint32_t issued = 0, done = 0;
      uint32_t head = 0, tail = 0;  // monotonic ring positions (the ring is empty between layers)
      while (done < ni) {
        // issue as many items as slots and ring bytes allow (warp-uniform decisions)
        while (issued < ni && issued - done < STREAM_SLOTS) {
          const uint32_t i = issued, r = wr.row0 + i * wr.stride;
          uint4 m;
          uint32_t dref;
          if (i < STREAM_DESC) {
            m = wa->dmeta[i];
            dref = wa->ddst[i];
          } else {
            m = __ldg(&d.meta[o0 + r]);
            dref = __ldg(&d.dst[o0 + r]);
          }
          const uint32_t ar = (m.w & CTL_EXT) ? 0u : (m.w >> 5) & 3u;
          const uint32_t b0 = ar ? CH << (m.x >> 30) : 0u, b1 = ar >= 2 ? CH << (m.y >> 30) : 0u,
                         b2 = ar >= 3 ? CH << (m.z >> 30) : 0u;
          const uint32_t need = b0 + b1 + b2;
          if (issued == done) head = tail = 0;  // nothing in flight: start the ring afresh (no wrap gap)
          uint32_t p = head;
          if ((p % STREAM_RING) + need > STREAM_RING) p = (p / STREAM_RING + 1u) * STREAM_RING;  // no wrap inside
          if (p + need - tail > STREAM_RING) break;                                            // ring full
          const uint32_t slot = (uses + i) % STREAM_SLOTS;
          if (lane_id == 0) {
            SlotInfo& si = wa->slot[slot];
            si.meta = m;
            si.dst = dref;
            si.off[0] = p % STREAM_RING;
            si.off[1] = (p + b0) % STREAM_RING;
            si.end = p + need;
            if (!need) {
              mbar_arrive(&wa->full[slot]);
            } else {
              mbar_arrive_expect_tx(&wa->full[slot], need);
              bulk_g2s(wa->ring + si.off[0], elem(s.state, m.x, s.n_pad, lane0), b0, &wa->full[slot]);
              if (b1) bulk_g2s(wa->ring + si.off[1], elem(s.state, m.y, s.n_pad, lane0), b1, &wa->full[slot]);
              if (b2) bulk_g2s(wa->ring + si.off[1] + b1, elem(s.state, m.z, s.n_pad, lane0), b2, &wa->full[slot]);
            }
          }
          head = p + need;
          issued++;
        }
        // consume the oldest item
        const uint32_t i = done, slot = (uses + i) % STREAM_SLOTS, par = ((uses + i) / STREAM_SLOTS) & 1u;
        int ok = 1;
        if (lane_id == 0) ok = mbar_wait(&wa->full[slot], par, g.timeout_ns) ? 1 : 0;
        ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
        if (!ok) {
          if (lane_id == 0) atomicOr(s.err, 2u);
          bad = true;
          break;
        }
        const SlotInfo& si = wa->slot[slot];
        stream_item<H>(d, s, si, wa->ring, lane0, lane_id, am);
        tail = si.end;
        __syncwarp();
        if (lane_id == 0) fence_proxy_async();  // the bytes just read may be overwritten by later copies
        done++;
      }
      if (bad) {
        // wait (bounded) for the copies this warp issued and has not consumed,
        // the timed-out item's included
        if (lane_id == 0)
          for (uint32_t i = done; i < issued; i++) {
            const uint32_t slot = (uses + i) % STREAM_SLOTS, par = ((uses + i) / STREAM_SLOTS) & 1u;
            if (!mbar_wait(&wa->full[slot], par, g.timeout_ns)) {
              atomicOr(s.err, 4u);
              break;
            }
          }
        __syncwarp();
        grid_sync(g, s.err, &sh_ok);
        return;
      }
      uses += ni;
      if (!grid_sync_staging(g, s.err, &sh_ok, [&] { stream_stage(d, L + 1u, wr, wa, lane_id); })) return;
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
