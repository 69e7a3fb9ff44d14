// flow_items.cuh -- the FLOW form's device functions (the evaluation phase of
// a cycle without barriers between layers; the kernel is in flow.cuh).  They
// need kernels.cuh and the few memory operations defined below, so a host
// compiler can run them too (the test harness does, one host thread per lane).
#pragma once
#include <cstddef>
#include <cstdint>
#ifndef __CUDA_ARCH__
#include <chrono>
#include <thread>
#endif

#include "flow_tables.hpp"
#include "kernels.cuh"

namespace rteaal {

struct FlowArgs {
  // [rows in layout order][n_pad] pairs of words: value bits 0..31 | stamp << 32,
  // value bits 32..63 | stamp << 32 (16 bytes, one vector store)
  unsigned long long* mirror;
  // per lowered op: {operand rows a, b, c (layout order; bit 31: written in the
  // cycle, so its stamp is checked), output row}, {ctl, output row reference,
  // side-array offset, operand count} -- the side array `fext` holding operand
  // rows with the same flag for ops with more than three operands
  const uint4* fop;
  const uint32_t* fext;
  // rows read but not written in the cycle: [inputs, registers, constants]
  // as {row reference, row}
  const uint2* fpool;
  uint32_t n_in, n_reg, n_const;
  uint32_t epoch;       // cycle c of the launch stamps its results epoch + c + 1
  uint32_t skew;        // 0; a test hook makes items wait for a stamp that never comes
  uint64_t timeout_ns;  // bound of every stamp wait (the launch's barriers wait twice as long)
  int off_in_smem;      // the launch's dynamic shared memory holds the layer offsets
  uint32_t kw;          // items a warp takes per layer and round (its first kw lanes), 1..32
  FastDiv span;         // lanes the launch visits
};

// The memory operations the form needs: relaxed (gpu scope) 16-byte stores and
// loads of a pair of stamped words, a relaxed load of the error word and the
// global timer.  A host compiler (the test harness that runs this code on the
// CPU) gets the same semantics from per-word atomics and a steady clock.
__device__ __forceinline__ void st_relaxed_v2(unsigned long long* p, unsigned long long a, unsigned long long b) {
#ifdef __CUDA_ARCH__
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
#else
  __atomic_store_n(p, a, __ATOMIC_RELAXED);
  __atomic_store_n(p + 1, b, __ATOMIC_RELAXED);
#endif
}
__device__ __forceinline__ ulonglong2 ld_relaxed_v2(const unsigned long long* p) {
  ulonglong2 v;
#ifdef __CUDA_ARCH__
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
#else
  v.x = __atomic_load_n(p, __ATOMIC_RELAXED);
  v.y = __atomic_load_n(p + 1, __ATOMIC_RELAXED);
#endif
  return v;
}
__device__ __forceinline__ uint32_t flow_ld_err(const uint32_t* p) {
#ifdef __CUDA_ARCH__
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
#else
  return __atomic_load_n(p, __ATOMIC_RELAXED);
#endif
}
__device__ __forceinline__ uint64_t flow_clock() {
#ifdef __CUDA_ARCH__
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
#else
  std::this_thread::yield();  // a host thread that polls lets the others run
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
#endif
}

__device__ __forceinline__ unsigned long long* flow_word(const DSim& s, const FlowArgs& f, uint32_t row,
                                                         uint32_t lane) {
  return f.mirror + ((size_t)(row & ~FLOW_CHECK) * s.n_pad + lane) * 2u;
}

// The stamped words of an operand hold this cycle's value (or need no stamp).
__device__ __forceinline__ bool flow_ready(uint32_t row, const ulonglong2& w, uint32_t stamp) {
  return !(row & FLOW_CHECK) || ((uint32_t)(w.x >> 32) == stamp && (uint32_t)(w.y >> 32) == stamp);
}

__device__ __forceinline__ uint64_t flow_take(const ulonglong2& w) {
  return (w.x & 0xFFFFFFFFull) | (w.y << 32);
}

// Copy rows [i0, i1) of the pool list from the compact state to their words:
// the (row, lane) pairs this thread's ItemSpace gives (the ones it wrote itself
// in the stimulus or the clock edge).
__device__ __forceinline__ void flow_refresh(const DSim& s, const FlowArgs& f, const ItemSpace& is, uint32_t i0,
                                             uint32_t i1) {
  for_rows<1>(is, i1 - i0, [&](uint32_t j, uint32_t lane) {
    const uint2 e = __ldg(&f.fpool[i0 + j]);
    const uint64_t v = ld1(s.state, e.x, s.n_pad, lane);
    st_relaxed_v2(flow_word(s, f, e.y, lane), v & 0xFFFFFFFFull, v >> 32);
  });
}

// One operand of an extended op, waited for on its own.
__device__ __forceinline__ bool flow_value(const DSim& s, const FlowArgs& f, uint32_t row, uint32_t lane,
                                           uint32_t stamp, uint64_t timeout_ns, uint64_t& v) {
  const unsigned long long* w = flow_word(s, f, row, lane);
  ulonglong2 x = ld_relaxed_v2(w);
  if (!flow_ready(row, x, stamp)) {
    const uint64_t t0 = flow_clock();
    do {
      if (flow_ld_err(s.err) != 0u) return false;
      if (flow_clock() - t0 > timeout_ns) {
        atomicOr(s.err, 8u);
        return false;
      }
      x = ld_relaxed_v2(w);
    } while (!flow_ready(row, x, stamp));
  }
  v = flow_take(x);
  return true;
}

// One item per lane of a warp -- a lowered op (descriptor q) for one lane:
// op_u / op_r / op_s of Cascade 1; `has` false: the lane has no item.  Every
// operand is one 16-byte load of its words, issued before any is used (by
// flow_issue, while the warp finished its previous item).  The warp waits as
// one: its lanes with at most three operands reload the operands
// not yet stamped until every such lane has all of them (a spinning lane never
// diverges from the others); lanes of extended ops wait operand by operand.
// Returns false if a wait gave up (then the error word is set).
__device__ __forceinline__ bool flow_items(const DDesign& d, const DSim& s, const FlowArgs& f, bool has,
                                           const uint4& qa, const uint4& qb, uint32_t lane, ulonglong2 wa,
                                           ulonglong2 wb, ulonglong2 wc, uint32_t stamp, uint32_t want,
                                           uint64_t timeout_ns) {
  const uint32_t ctl = qb.x;
  const bool ext = has && (ctl & CTL_EXT);
  const uint32_t plain = __ballot_sync(0xFFFFFFFFu, has && !ext);  // lanes that wait together
  bool ok = true;
  uint64_t r = 0;
  if (ext) {  // more than three operands: one after another from the side array
    const Lanes<1> x = ext_eval<1, Lanes<1>>(f.fext + qb.z, ctl & 31u, qb.w, [&](uint32_t row) {
      Lanes<1> y;
      y.x[0] = 0ull;
      if (ok) ok = flow_value(s, f, row, lane, want, timeout_ns, y.x[0]);
      return y;
    });
    r = x.x[0] & wmask(ctl_width(ctl));
  } else if (has) {
    const uint32_t ar = (ctl >> 5) & 3u;
    const uint32_t rb = ar >= 2 ? qa.y : 0u, rc = ar >= 3 ? qa.z : 0u;  // row 0 unchecked: a spare load
    auto ready = [&] {
      return flow_ready(qa.x, wa, want) && flow_ready(rb, wb, want) && flow_ready(rc, wc, want);
    };
    if (!__all_sync(plain, ready())) {
      const uint64_t t0 = flow_clock();
      uint32_t it = 0;
      do {
        if ((++it & 15u) == 0u) {
          bool stop = flow_ld_err(s.err) != 0u;
          if (!stop && flow_clock() - t0 > timeout_ns) {
            atomicOr(s.err, 8u);
            stop = true;
          }
          if (__any_sync(plain, stop)) {
            ok = false;
            break;
          }
        }
        if (!flow_ready(qa.x, wa, want)) wa = ld_relaxed_v2(flow_word(s, f, qa.x, lane));
        if (!flow_ready(rb, wb, want)) wb = ld_relaxed_v2(flow_word(s, f, rb, lane));
        if (!flow_ready(rc, wc, want)) wc = ld_relaxed_v2(flow_word(s, f, rc, lane));
      } while (!__all_sync(plain, ready()));
    }
    if (ok) {
      const uint64_t a = flow_take(wa), b = flow_take(wb), c = flow_take(wc);
      r = (ctl & 31u) == OP_MEMRD ? eval_memrd(d, s, ctl, a, lane) : alu(ctl, a, b, c);
    }
  }
  if (has && ok) {  // the stamped words first (others wait on them), then the compact row
    const unsigned long long sv = (unsigned long long)stamp << 32;
    st_relaxed_v2(flow_word(s, f, qa.w, lane), (r & 0xFFFFFFFFull) | sv, (r >> 32) | sv);
    st1(s.state, qb.y, s.n_pad, lane, r);
  }
  return __all_sync(0xFFFFFFFFu, ok);
}

// The operand words of an item with at most three operands, loaded ahead:
// those written earlier (most of an item's operands, once its producers are
// done) are then ready when the item is evaluated; the others are reloaded.
__device__ __forceinline__ void flow_issue(const DSim& s, const FlowArgs& f, bool has, const uint4& qa,
                                           const uint4& qb, uint32_t lane, ulonglong2& wa, ulonglong2& wb,
                                           ulonglong2& wc) {
  const uint32_t ar = (qb.x >> 5) & 3u;
  const bool plain = has && !(qb.x & CTL_EXT);
  wa = ld_relaxed_v2(flow_word(s, f, plain ? qa.x : 0u, lane));
  wb = ld_relaxed_v2(flow_word(s, f, plain && ar >= 2 ? qa.y : 0u, lane));
  wc = ld_relaxed_v2(flow_word(s, f, plain && ar >= 3 ? qa.z : 0u, lane));
}

// A warp's position in the evaluation phase: layer L (rows from o0, n items)
// and the item index of its first thread (warp w takes items w kw .. w kw +
// kw - 1, then the same plus W kw, ... for W warps: fewer items per warp than
// lanes make a warp wait for fewer producers).
struct FlowPos {
  uint32_t L, o0, n, base;
};

// Move to the warp's next position with items (base + T in this layer, else
// the first later layer that has items for it); false past the last layer.
__device__ __forceinline__ bool flow_next(const DDesign& d, const FlowArgs& f, const uint32_t* off, FlowPos& p,
                                          uint32_t t0, uint32_t T) {
  p.base += T;  // T: items of one round (warps x kw)
  while (p.base >= p.n) {
    if (++p.L >= d.n_layers) return false;
    p.o0 = off[p.L];
    p.n = (off[p.L + 1] - p.o0) * f.span.d;
    p.base = t0;
  }
  return true;
}

// One lane's item at a position: its descriptor, loaded one position ahead of
// its evaluation (it depends on no result).
struct FlowSlot {
  uint4 qa, qb;
  uint32_t lane;
  bool has;
};

__device__ __forceinline__ FlowSlot flow_slot(const DSim& s, const FlowArgs& f, const FlowPos& p, uint32_t t,
                                              uint32_t c) {
  FlowSlot q{make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), 0u, false};
  const uint32_t i = p.base + (t & 31u);
  if ((t & 31u) < f.kw && i < p.n) {
    const uint32_t r = fdiv(f.span, i);
    q.lane = i - r * f.span.d;
    q.has = lane_active(s, q.lane, c);  // a frozen lane's results are read only by itself
    if (q.has) {
      q.qa = __ldg(&f.fop[2 * (p.o0 + r)]);
      q.qb = __ldg(&f.fop[2 * (p.o0 + r) + 1]);
    }
  }
  return q;
}

// The evaluation phase of cycle c: the warps take the items of every layer in
// turn (an item being (row, lane), the lanes of a row adjacent), kw per warp
// and round; a warp's threads go through their items together.  `off`: the
// layer offsets (in shared memory when they fit).
__device__ __forceinline__ bool flow_cycle(const DDesign& d, const DSim& s, const FlowArgs& f, const uint32_t* off,
                                           uint32_t c, uint32_t t, uint32_t T, uint64_t timeout_ns) {
  const uint32_t stamp = f.epoch + c + 1u, t0 = (t >> 5) * f.kw, R = (T >> 5) * f.kw;
  FlowPos p{0u, 0u, 0u, t0};
  bool more = false;
  if (d.n_layers > 0) {
    p.o0 = off[0];
    p.n = (off[1] - p.o0) * f.span.d;
    more = p.base < p.n || flow_next(d, f, off, p, t0, R);
  }
  FlowSlot cur = more ? flow_slot(s, f, p, t, c) : FlowSlot{};
  ulonglong2 wa, wb, wc;
  flow_issue(s, f, cur.has, cur.qa, cur.qb, cur.lane, wa, wb, wc);
  while (more) {
    FlowPos pn = p;
    more = flow_next(d, f, off, pn, t0, R);
    const FlowSlot nx = more ? flow_slot(s, f, pn, t, c) : FlowSlot{};
    if (!flow_items(d, s, f, cur.has, cur.qa, cur.qb, cur.lane, wa, wb, wc, stamp, stamp + f.skew, timeout_ns))
      return false;
    p = pn;
    cur = nx;
    flow_issue(s, f, cur.has, cur.qa, cur.qb, cur.lane, wa, wb, wc);
  }
  return true;
}

}  // namespace rteaal
