// kernels.cuh -- sm_103a kernels of one simulated cycle.
//
// State layout: one row per signal, lane-minor (lane = stimulus instance), each
// row stored at its width class -- 1, 2, 4 or 8 bytes per lane for widths up to
// 8, 16, 32, 64 -- since every value is kept masked to its width.  Rows are
// addressed by 32-bit references (class, per-lane byte offset); values are
// widened to 64 bits only in registers.  One "item" is one operation evaluated
// for V consecutive lanes; the lanes of an operation are spread over
// consecutive threads, so a warp reads one contiguous segment of each operand
// row (coalesced) and the operation's descriptor is a broadcast read.
// Operations of a layer are stored grouped by (opcode, width), so neighbouring
// threads take the same switch arm.  No tensor cores: this is integer gather
// work bound by memory.
#pragma once
#include <cstdint>

#include "lower.hpp"

namespace rteaal {

struct DDesign {
  const uint4* meta;          // [n_lowered] {a, b, c, ctl}, operands as row references
  const uint32_t* dst;        // [n_lowered] row reference of each op's output
  const uint32_t* ext;        // operand row references of ops with > 3 operands
  const uint32_t* layer_off;  // [n_layers + 1]
  const uint32_t* layer_ext;  // [n_layers] first op with > 3 operands (they close each layer)
  const uint32_t* layer_wide; // [n_layers] first op with <= 3 operands that is not narrow
  const uint32_t* reg_src;    // [n_regs] row reference of D
  const uint32_t* reg_ref;    // [n_regs] row reference of Q
  const uint32_t* reg_w;      // [n_regs]
  const uint64_t* reg_init;   // [n_regs]
  const uint4* wport;         // [n_wports] {mem, en, addr, data} grouped by memory
  const uint4* mem_info;      // [n_mems + 1] {word offset, words-1, width, first port}
  const uint32_t* in_w;       // [n_inputs]
  const uint32_t* in_ref;     // [n_inputs]
  uint32_t n_layers, n_regs, n_inputs, n_mems, op_base, reg_base;
  uint4 cls_off;              // per class k: first per-lane byte offset of the class's rows
  uint4 cls_idx;              // per class k: index of the class's first row (rows in layout order)
};

// Divide by a runtime constant with a multiply-high (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Fig. 4.1):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, q = (mulhi(m, n) + n) >> l.
struct FastDiv {
  uint32_t d, m, l;
};

__host__ __device__ inline uint32_t fdiv(const FastDiv& f, uint32_t n) {
#ifdef __CUDA_ARCH__
  const uint64_t t = __umulhi(n, f.m);
#else
  const uint64_t t = ((uint64_t)n * f.m) >> 32;
#endif
  return (uint32_t)((t + n) >> f.l);
}

struct DSim {
  uint8_t* state;               // compact rows, see above
  uint64_t* mem;
  uint64_t* xs;                 // [n_inputs][n_pad] xorshift64 states
  uint32_t n_pad, n_user;
  const uint32_t* budget;       // [n_pad] cycles this step, or null -> uniform
  uint32_t uniform;
  const uint32_t* user_of_lane; // null = identity
  int stim_mode;
  const uint64_t* stim;         // [cycles][n_inputs][n_user]
  int reset;
  const uint32_t* reset_lane;   // [n_pad] leading reset cycles per lane, or null
  const uint32_t* probe_slot;   // EVERY / CHANGES probes (row references)
  uint32_t n_probe;
  uint64_t* probe_out;          // EVERY: [cycles][n_probe][n_user]; CHANGES: records
  int probe_changes;            // CHANGES mode
  uint64_t* probe_prev;         // CHANGES: [n_probe][n_pad] previous values
  unsigned long long* change_count;
  uint64_t change_cap;
  uint32_t* err;
  // activity-aware evaluation (null act: off).  act[row][chunk] = low 8 bits
  // of the last cycle in which the row changed in any lane of the 128-lane
  // chunk; cycle numbers count from the sim's creation (act_g0 = this step's
  // first).  act_force: the step's first cycle evaluates every op.
  uint8_t* act;
  uint32_t act_chunks, act_g0;
  int act_force;
  unsigned long long* act_count;  // [2]: items evaluated, items skipped
};

constexpr uint32_t NO_ROW = 0xFFFFFFFFu;

// Work of one thread over a lane range [lane_base, lane_base + tpo * V): rows
// (operations, inputs, registers, ...) times chunks of V lanes.
//  * fixed mapping (row_stride != 0): when the threads cover every chunk, each
//    thread keeps one chunk and walks rows row0, row0 + row_stride, ...  No
//    division per item and the lane activity is computed once per phase.
//  * generic mapping (row_stride == 0): item i = first + k * stride,
//    row = i / tpo, chunk = i % tpo (fewer threads than chunks).
struct ItemSpace {
  FastDiv tpo;
  uint32_t lane_base;
  uint32_t first, stride;
  uint32_t lane, row0, row_stride;
};

template <int V>
__device__ __forceinline__ ItemSpace make_space(FastDiv tpo, uint32_t lane_base, uint32_t t,
                                                uint32_t nthreads) {
  ItemSpace is;
  is.tpo = tpo;
  is.lane_base = lane_base;
  is.first = t;
  is.stride = nthreads;
  is.lane = lane_base;
  is.row0 = NO_ROW;
  is.row_stride = 0;
  if (nthreads >= tpo.d) {
    const uint32_t per = fdiv(tpo, nthreads);
    is.row_stride = per;
    if (t < per * tpo.d) {
      const uint32_t r = fdiv(tpo, t);
      is.row0 = r;
      is.lane = lane_base + (t - r * tpo.d) * V;
    }
  }
  return is;
}

__device__ __forceinline__ uint64_t wmask(uint32_t w) { return ~0ull >> (64u - w); }

__device__ __forceinline__ bool lane_active(const DSim& s, uint32_t lane, uint32_t cyc) {
  return s.budget ? cyc < __ldg(&s.budget[lane]) : (lane < s.n_user && cyc < s.uniform);
}

__device__ __forceinline__ uint32_t user_of(const DSim& s, uint32_t lane) {
  return s.user_of_lane ? __ldg(&s.user_of_lane[lane]) : lane;
}

// Every opcode except MEMRD and the extended-operand form, then masked to width.
__device__ __forceinline__ uint64_t alu(uint32_t ctl, uint64_t a, uint64_t b, uint64_t c) {
  const uint32_t op = ctl & 31u, ar = (ctl >> 5) & 3u;
  const uint32_t p0 = (ctl >> 16) & 255u, p1 = ctl >> 24;
  uint64_t r;
  switch (op) {
    case OP_COPY: r = a; break;
    case OP_AND: r = a & b; if (ar == 3) r &= c; break;
    case OP_OR: r = a | b; if (ar == 3) r |= c; break;
    case OP_XOR: r = a ^ b; if (ar == 3) r ^= c; break;
    case OP_NOT: r = ~a; break;
    case OP_ADD: r = a + b; if (ar == 3) r += c; break;
    case OP_SUB: r = a - b; break;
    case OP_MUL: r = a * b; if (ar == 3) r *= c; break;
    case OP_SHL: r = p0 >= 64u ? 0ull : a << p0; break;
    case OP_SHR: r = p0 >= 64u ? 0ull : a >> p0; break;
    case OP_DSHL: r = b >= 64ull ? 0ull : a << (uint32_t)b; break;
    case OP_DSHR: r = b >= 64ull ? 0ull : a >> (uint32_t)b; break;
    case OP_BITS: r = (a >> p1) & wmask(p0 - p1 + 1u); break;
    case OP_CAT: r = (p0 >= 64u ? 0ull : a << p0) | b; break;
    case OP_EQ: r = a == b; break;
    case OP_NEQ: r = a != b; break;
    case OP_LT: r = a < b; break;
    case OP_LEQ: r = a <= b; break;
    case OP_GT: r = a > b; break;
    case OP_GEQ: r = a >= b; break;
    case OP_MUX: r = (a & 1ull) ? b : c; break;
    case OP_ANDR: { const uint64_t m = wmask(p0); r = (a & m) == m; } break;
    case OP_ORR: r = a != 0ull; break;
    case OP_XORR: r = (uint64_t)(__popcll(a) & 1); break;
    default: r = 0; break;
  }
  return r & wmask(ctl_width(ctl));
}

// Address of element (row, lane) of the compact state.
__device__ __forceinline__ const uint8_t* elem(const uint8_t* st, uint32_t ref, size_t np,
                                               uint32_t lane) {
  // one 32 x 32 -> 64-bit multiply-add; lane << class fits 32 bits
  return st + ((uint64_t)(ref & REF_OFF_MASK) * (uint32_t)np + (uint32_t)(lane << (ref >> 30)));
}

// Index of a row in layout order (class 3 rows first), from its reference.
__device__ __forceinline__ uint32_t row_index(const DDesign& d, uint32_t ref) {
  const uint32_t k = ref >> 30;
  const uint32_t off = k == 0 ? d.cls_off.x : k == 1 ? d.cls_off.y : k == 2 ? d.cls_off.z : d.cls_off.w;
  const uint32_t idx = k == 0 ? d.cls_idx.x : k == 1 ? d.cls_idx.y : k == 2 ? d.cls_idx.z : d.cls_idx.w;
  return idx + (((ref & REF_OFF_MASK) - off) >> k);
}

// Activity stamp of (row, 128-lane chunk).
__device__ __forceinline__ uint8_t* act_at(const DDesign& d, const DSim& s, uint32_t ref, uint32_t lane) {
  return s.act + (size_t)row_index(d, ref) * s.act_chunks + (lane >> 7);
}

// one element, zero-extended
__device__ __forceinline__ uint64_t ld1(const uint8_t* st, uint32_t ref, size_t np, uint32_t lane) {
  const uint8_t* p = elem(st, ref, np, lane);
  switch (ref >> 30) {
    case 0: return *p;
    case 1: return *reinterpret_cast<const uint16_t*>(p);
    case 2: return *reinterpret_cast<const uint32_t*>(p);
    default: return *reinterpret_cast<const uint64_t*>(p);
  }
}

// one element (the value already fits its row's class)
__device__ __forceinline__ void st1(uint8_t* st, uint32_t ref, size_t np, uint32_t lane, uint64_t v) {
  uint8_t* p = const_cast<uint8_t*>(elem(st, ref, np, lane));
  switch (ref >> 30) {
    case 0: *p = (uint8_t)v; break;
    case 1: *reinterpret_cast<uint16_t*>(p) = (uint16_t)v; break;
    case 2: *reinterpret_cast<uint32_t*>(p) = (uint32_t)v; break;
    default: *reinterpret_cast<uint64_t*>(p) = v; break;
  }
}

__device__ __forceinline__ uint64_t eval_memrd(const DDesign& d, const DSim& s, uint32_t ctl,
                                               uint64_t addr, uint32_t lane) {
  const uint32_t mi = ((ctl >> 16) & 255u) | ((ctl >> 24) << 8);
  const uint4 info = __ldg(&d.mem_info[mi]);
  const uint64_t v = s.mem[((size_t)info.x + (addr & (uint64_t)info.y)) * s.n_pad + lane];
  return v & wmask(ctl_width(ctl));
}

template <int V>
struct Lanes {
  uint64_t x[V];
};

// alu for V lanes with one opcode dispatch per item (the lane loop is inside
// each case), then the width mask.
template <int V>
__device__ __forceinline__ Lanes<V> alu_v(uint32_t ctl, const Lanes<V>& a, const Lanes<V>& b,
                                          const Lanes<V>& c) {
  const uint32_t op = ctl & 31u, ar = (ctl >> 5) & 3u;
  const uint32_t p0 = (ctl >> 16) & 255u, p1 = ctl >> 24;
  Lanes<V> r;
#define RT_LANES(expr) _Pragma("unroll") for (int v = 0; v < V; v++) r.x[v] = (expr)
  switch (op) {
    case OP_COPY: RT_LANES(a.x[v]); break;
    case OP_AND: RT_LANES(a.x[v] & b.x[v]); if (ar == 3) RT_LANES(r.x[v] & c.x[v]); break;
    case OP_OR: RT_LANES(a.x[v] | b.x[v]); if (ar == 3) RT_LANES(r.x[v] | c.x[v]); break;
    case OP_XOR: RT_LANES(a.x[v] ^ b.x[v]); if (ar == 3) RT_LANES(r.x[v] ^ c.x[v]); break;
    case OP_NOT: RT_LANES(~a.x[v]); break;
    case OP_ADD: RT_LANES(a.x[v] + b.x[v]); if (ar == 3) RT_LANES(r.x[v] + c.x[v]); break;
    case OP_SUB: RT_LANES(a.x[v] - b.x[v]); break;
    case OP_MUL: RT_LANES(a.x[v] * b.x[v]); if (ar == 3) RT_LANES(r.x[v] * c.x[v]); break;
    case OP_SHL: RT_LANES(p0 >= 64u ? 0ull : a.x[v] << p0); break;
    case OP_SHR: RT_LANES(p0 >= 64u ? 0ull : a.x[v] >> p0); break;
    case OP_DSHL: RT_LANES(b.x[v] >= 64ull ? 0ull : a.x[v] << (uint32_t)b.x[v]); break;
    case OP_DSHR: RT_LANES(b.x[v] >= 64ull ? 0ull : a.x[v] >> (uint32_t)b.x[v]); break;
    case OP_BITS: {
      const uint64_t m = wmask(p0 - p1 + 1u);
      RT_LANES((a.x[v] >> p1) & m);
    } break;
    case OP_CAT: RT_LANES((p0 >= 64u ? 0ull : a.x[v] << p0) | b.x[v]); break;
    case OP_EQ: RT_LANES((uint64_t)(a.x[v] == b.x[v])); break;
    case OP_NEQ: RT_LANES((uint64_t)(a.x[v] != b.x[v])); break;
    case OP_LT: RT_LANES((uint64_t)(a.x[v] < b.x[v])); break;
    case OP_LEQ: RT_LANES((uint64_t)(a.x[v] <= b.x[v])); break;
    case OP_GT: RT_LANES((uint64_t)(a.x[v] > b.x[v])); break;
    case OP_GEQ: RT_LANES((uint64_t)(a.x[v] >= b.x[v])); break;
    case OP_MUX: RT_LANES((a.x[v] & 1ull) ? b.x[v] : c.x[v]); break;
    case OP_ANDR: {
      const uint64_t m = wmask(p0);
      RT_LANES((uint64_t)((a.x[v] & m) == m));
    } break;
    case OP_ORR: RT_LANES((uint64_t)(a.x[v] != 0ull)); break;
    case OP_XORR: RT_LANES((uint64_t)(__popcll(a.x[v]) & 1)); break;
    default: RT_LANES(0ull); break;
  }
#undef RT_LANES
  const uint64_t mk = wmask(ctl_width(ctl));
#pragma unroll
  for (int v = 0; v < V; v++) r.x[v] &= mk;
  return r;
}

// V consecutive lanes of a row, zero-extended (lane is a multiple of V, so the
// packed 2^k * V bytes are naturally aligned).
template <int V>
__device__ __forceinline__ Lanes<V> ldr(const uint8_t* st, uint32_t ref, size_t np, uint32_t lane) {
  Lanes<V> r;
  if constexpr (V == 2) {
    const uint8_t* p = elem(st, ref, np, lane);
    switch (ref >> 30) {
      case 0: {
        const uint32_t t = *reinterpret_cast<const uint16_t*>(p);
        r.x[0] = t & 0xFFu;
        r.x[1] = t >> 8;
      } break;
      case 1: {
        const uint32_t t = *reinterpret_cast<const uint32_t*>(p);
        r.x[0] = t & 0xFFFFu;
        r.x[1] = t >> 16;
      } break;
      case 2: {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        r.x[0] = t.x;
        r.x[1] = t.y;
      } break;
      default: {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(p);
        r.x[0] = t.x;
        r.x[1] = t.y;
      } break;
    }
  } else if constexpr (V == 4) {
    const uint8_t* p = elem(st, ref, np, lane);
    switch (ref >> 30) {
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
  } else if constexpr (V == 8) {
    const uint8_t* p = elem(st, ref, np, lane);
    switch (ref >> 30) {
      case 0: {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
#pragma unroll
        for (int v = 0; v < 4; v++) {
          r.x[v] = (t.x >> (8 * v)) & 0xFFu;
          r.x[4 + v] = (t.y >> (8 * v)) & 0xFFu;
        }
      } break;
      case 1: {
        const uint4 t = *reinterpret_cast<const uint4*>(p);
        r.x[0] = t.x & 0xFFFFu; r.x[1] = t.x >> 16;
        r.x[2] = t.y & 0xFFFFu; r.x[3] = t.y >> 16;
        r.x[4] = t.z & 0xFFFFu; r.x[5] = t.z >> 16;
        r.x[6] = t.w & 0xFFFFu; r.x[7] = t.w >> 16;
      } break;
      case 2: {
        const uint4 t0 = reinterpret_cast<const uint4*>(p)[0];
        const uint4 t1 = reinterpret_cast<const uint4*>(p)[1];
        r.x[0] = t0.x; r.x[1] = t0.y; r.x[2] = t0.z; r.x[3] = t0.w;
        r.x[4] = t1.x; r.x[5] = t1.y; r.x[6] = t1.z; r.x[7] = t1.w;
      } break;
      default: {
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const ulonglong2 t = reinterpret_cast<const ulonglong2*>(p)[q];
          r.x[2 * q] = t.x;
          r.x[2 * q + 1] = t.y;
        }
      } break;
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; v++) r.x[v] = ld1(st, ref, np, lane + v);
  }
  return r;
}

// ---- narrow ops (CTL_NARROW): operands and result of at most 32 bits, so the
// whole item stays in 32-bit registers: half the registers, and one
// instruction per lane where 64-bit arithmetic takes two.
template <int V>
struct Lanes32 {
  uint32_t x[V];
};

__device__ __forceinline__ uint32_t wmask32(uint32_t w) { return 0xFFFFFFFFu >> (32u - w); }

// V consecutive lanes of a row of class 0, 1 or 2, zero-extended to 32 bits.
template <int V>
__device__ __forceinline__ Lanes32<V> ldr32(const uint8_t* st, uint32_t ref, size_t np, uint32_t lane) {
  Lanes32<V> r;
  const uint8_t* p = elem(st, ref, np, lane);
  const uint32_t k = ref >> 30;
  if constexpr (V == 4) {
    if (k == 0) {
      const uint32_t t = *reinterpret_cast<const uint32_t*>(p);
#pragma unroll
      for (int v = 0; v < 4; v++) r.x[v] = __byte_perm(t, 0u, 0x4440u + v);
    } else if (k == 1) {
      const uint2 t = *reinterpret_cast<const uint2*>(p);
      r.x[0] = t.x & 0xFFFFu; r.x[1] = t.x >> 16;
      r.x[2] = t.y & 0xFFFFu; r.x[3] = t.y >> 16;
    } else {
      const uint4 t = *reinterpret_cast<const uint4*>(p);
      r.x[0] = t.x; r.x[1] = t.y; r.x[2] = t.z; r.x[3] = t.w;
    }
  } else if constexpr (V == 8) {
    if (k == 0) {
      const uint2 t = *reinterpret_cast<const uint2*>(p);
#pragma unroll
      for (int v = 0; v < 4; v++) {
        r.x[v] = __byte_perm(t.x, 0u, 0x4440u + v);
        r.x[4 + v] = __byte_perm(t.y, 0u, 0x4440u + v);
      }
    } else if (k == 1) {
      const uint4 t = *reinterpret_cast<const uint4*>(p);
      r.x[0] = t.x & 0xFFFFu; r.x[1] = t.x >> 16;
      r.x[2] = t.y & 0xFFFFu; r.x[3] = t.y >> 16;
      r.x[4] = t.z & 0xFFFFu; r.x[5] = t.z >> 16;
      r.x[6] = t.w & 0xFFFFu; r.x[7] = t.w >> 16;
    } else {
      const uint4 t0 = reinterpret_cast<const uint4*>(p)[0];
      const uint4 t1 = reinterpret_cast<const uint4*>(p)[1];
      r.x[0] = t0.x; r.x[1] = t0.y; r.x[2] = t0.z; r.x[3] = t0.w;
      r.x[4] = t1.x; r.x[5] = t1.y; r.x[6] = t1.z; r.x[7] = t1.w;
    }
  } else if constexpr (V == 2) {
    if (k == 0) {
      const uint32_t t = *reinterpret_cast<const uint16_t*>(p);
      r.x[0] = t & 0xFFu; r.x[1] = t >> 8;
    } else if (k == 1) {
      const uint32_t t = *reinterpret_cast<const uint32_t*>(p);
      r.x[0] = t & 0xFFFFu; r.x[1] = t >> 16;
    } else {
      const uint2 t = *reinterpret_cast<const uint2*>(p);
      r.x[0] = t.x; r.x[1] = t.y;
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; v++) r.x[v] = (uint32_t)ld1(st, ref, np, lane + v);
  }
  return r;
}

// Store the active lanes (mask bit v = lane + v) of a narrow result (class 0..2).
template <int V>
__device__ __forceinline__ void str32(uint8_t* st, uint32_t ref, size_t np, uint32_t lane,
                                      const Lanes32<V>& r, uint32_t m) {
  uint8_t* p = const_cast<uint8_t*>(elem(st, ref, np, lane));
  const uint32_t k = ref >> 30;
  if constexpr (V == 4) {
    if (m == 15u) {
      if (k == 0)
        *reinterpret_cast<uint32_t*>(p) = r.x[0] | (r.x[1] << 8) | (r.x[2] << 16) | (r.x[3] << 24);
      else if (k == 1)
        *reinterpret_cast<uint2*>(p) = make_uint2(r.x[0] | (r.x[1] << 16), r.x[2] | (r.x[3] << 16));
      else
        *reinterpret_cast<uint4*>(p) = make_uint4(r.x[0], r.x[1], r.x[2], r.x[3]);
      return;
    }
  } else if constexpr (V == 8) {
    if (m == 255u) {
      if (k == 0) {
        *reinterpret_cast<uint2*>(p) =
            make_uint2(r.x[0] | (r.x[1] << 8) | (r.x[2] << 16) | (r.x[3] << 24),
                       r.x[4] | (r.x[5] << 8) | (r.x[6] << 16) | (r.x[7] << 24));
      } else if (k == 1) {
        *reinterpret_cast<uint4*>(p) = make_uint4(r.x[0] | (r.x[1] << 16), r.x[2] | (r.x[3] << 16),
                                                  r.x[4] | (r.x[5] << 16), r.x[6] | (r.x[7] << 16));
      } else {
        reinterpret_cast<uint4*>(p)[0] = make_uint4(r.x[0], r.x[1], r.x[2], r.x[3]);
        reinterpret_cast<uint4*>(p)[1] = make_uint4(r.x[4], r.x[5], r.x[6], r.x[7]);
      }
      return;
    }
  } else if constexpr (V == 2) {
    if (m == 3u) {
      if (k == 0) *reinterpret_cast<uint16_t*>(p) = (uint16_t)(r.x[0] | (r.x[1] << 8));
      else if (k == 1) *reinterpret_cast<uint32_t*>(p) = r.x[0] | (r.x[1] << 16);
      else *reinterpret_cast<uint2*>(p) = make_uint2(r.x[0], r.x[1]);
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < V; v++)
    if (m & (1u << v)) st1(st, ref, np, lane + v, r.x[v]);
}

// alu_v in 32-bit arithmetic for narrow ops.  Exactness against the 64-bit
// definition, with every operand < 2^32 and the result masked to w <= 32 bits:
// +, -, *, ~, &, |, ^ agree mod 2^32; shifting left by 32 or more leaves no
// bit below 32, shifting a 32-bit value right by 32 or more leaves 0 (so both
// give 0, here explicitly); BITS has hi < 32 and ANDR p0 <= 32 (lowering).
template <int V>
__device__ __forceinline__ Lanes32<V> alu32_v(uint32_t ctl, const Lanes32<V>& a, const Lanes32<V>& b,
                                              const Lanes32<V>& c) {
  const uint32_t op = ctl & 31u, ar = (ctl >> 5) & 3u;
  const uint32_t p0 = (ctl >> 16) & 255u, p1 = ctl >> 24;
  Lanes32<V> r;
#define RT_LANES(expr) _Pragma("unroll") for (int v = 0; v < V; v++) r.x[v] = (expr)
  switch (op) {
    case OP_COPY: RT_LANES(a.x[v]); break;
    case OP_AND: RT_LANES(a.x[v] & b.x[v]); if (ar == 3) RT_LANES(r.x[v] & c.x[v]); break;
    case OP_OR: RT_LANES(a.x[v] | b.x[v]); if (ar == 3) RT_LANES(r.x[v] | c.x[v]); break;
    case OP_XOR: RT_LANES(a.x[v] ^ b.x[v]); if (ar == 3) RT_LANES(r.x[v] ^ c.x[v]); break;
    case OP_NOT: RT_LANES(~a.x[v]); break;
    case OP_ADD: RT_LANES(a.x[v] + b.x[v]); if (ar == 3) RT_LANES(r.x[v] + c.x[v]); break;
    case OP_SUB: RT_LANES(a.x[v] - b.x[v]); break;
    case OP_MUL: RT_LANES(a.x[v] * b.x[v]); if (ar == 3) RT_LANES(r.x[v] * c.x[v]); break;
    case OP_SHL: RT_LANES(p0 >= 32u ? 0u : a.x[v] << p0); break;
    case OP_SHR: RT_LANES(p0 >= 32u ? 0u : a.x[v] >> p0); break;
    case OP_DSHL: RT_LANES(b.x[v] >= 32u ? 0u : a.x[v] << b.x[v]); break;
    case OP_DSHR: RT_LANES(b.x[v] >= 32u ? 0u : a.x[v] >> b.x[v]); break;
    case OP_BITS: {
      const uint32_t m = wmask32(p0 - p1 + 1u);
      RT_LANES((a.x[v] >> p1) & m);
    } break;
    case OP_CAT: RT_LANES((p0 >= 32u ? 0u : a.x[v] << p0) | b.x[v]); break;
    case OP_EQ: RT_LANES((uint32_t)(a.x[v] == b.x[v])); break;
    case OP_NEQ: RT_LANES((uint32_t)(a.x[v] != b.x[v])); break;
    case OP_LT: RT_LANES((uint32_t)(a.x[v] < b.x[v])); break;
    case OP_LEQ: RT_LANES((uint32_t)(a.x[v] <= b.x[v])); break;
    case OP_GT: RT_LANES((uint32_t)(a.x[v] > b.x[v])); break;
    case OP_GEQ: RT_LANES((uint32_t)(a.x[v] >= b.x[v])); break;
    case OP_MUX: RT_LANES((a.x[v] & 1u) ? b.x[v] : c.x[v]); break;
    case OP_ANDR: {
      const uint32_t m = wmask32(p0);
      RT_LANES((uint32_t)((a.x[v] & m) == m));
    } break;
    case OP_ORR: RT_LANES((uint32_t)(a.x[v] != 0u)); break;
    case OP_XORR: RT_LANES((uint32_t)(__popc(a.x[v]) & 1)); break;
    default: RT_LANES(0u); break;
  }
#undef RT_LANES
  const uint32_t mk = wmask32(ctl_width(ctl));
#pragma unroll
  for (int v = 0; v < V; v++) r.x[v] &= mk;
  return r;
}

// Ops with more than three operands (long mux chains from operator fusion,
// variadic folds), V lanes at a time: every operand row is one packed load.
// LT is Lanes<V> (64-bit) or Lanes32<V> (narrow ops); ld(ref) loads a row.
template <int V, typename LT, typename Load>
__device__ __forceinline__ LT ext_eval(const uint32_t* a, uint32_t op, uint32_t n, Load&& ld) {
  LT r;
  if (op == OP_MUXCHAIN) {
    // first set selector wins: walk the pairs in O order, a lane keeps the
    // first value whose selector is set, else the default.  The first four
    // pairs are unrolled so their operand loads are issued together.
    const uint32_t pairs = (n - 1u) >> 1;
    r = ld(__ldg(&a[n - 1]));
    uint32_t done = 0;  // bit v: lane + v already decided
    auto pair = [&](uint32_t i) {
      const LT sel = ld(__ldg(&a[2 * i]));
      const LT val = ld(__ldg(&a[2 * i + 1]));
#pragma unroll
      for (int v = 0; v < V; v++) {
        const bool take = (sel.x[v] & 1u) && !((done >> v) & 1u);
        r.x[v] = take ? val.x[v] : r.x[v];
        done |= (uint32_t)(sel.x[v] & 1u) << v;
      }
    };
#pragma unroll
    for (int i = 0; i < 4; i++)
      if ((uint32_t)i < pairs) pair((uint32_t)i);
    for (uint32_t i = 4; i < pairs; i++) pair(i);
  } else {
    r = ld(__ldg(&a[0]));
    for (uint32_t i = 1; i < n; i++) {
      const LT x = ld(__ldg(&a[i]));
#pragma unroll
      for (int v = 0; v < V; v++) {
        switch (op) {
          case OP_AND: r.x[v] &= x.x[v]; break;
          case OP_OR: r.x[v] |= x.x[v]; break;
          case OP_XOR: r.x[v] ^= x.x[v]; break;
          case OP_ADD: r.x[v] += x.x[v]; break;
          case OP_MUL: r.x[v] *= x.x[v]; break;
          default: break;
        }
      }
    }
  }
  return r;
}

template <int V>
__device__ __forceinline__ Lanes<V> eval_ext_v(const DDesign& d, const DSim& s, uint4 m, uint32_t lane) {
  Lanes<V> r = ext_eval<V, Lanes<V>>(d.ext + m.x, m.w & 31u, m.y, [&](uint32_t ref) {
    return ldr<V>(s.state, ref, s.n_pad, lane);
  });
  const uint64_t mk = wmask(ctl_width(m.w));
#pragma unroll
  for (int v = 0; v < V; v++) r.x[v] &= mk;
  return r;
}

// The same in 32-bit arithmetic for narrow ops (operands and result <= 32
// bits; the folds agree mod 2^32, selection moves values unchanged).
template <int V>
__device__ __forceinline__ Lanes32<V> eval_ext32_v(const DDesign& d, const DSim& s, uint4 m,
                                                   uint32_t lane) {
  Lanes32<V> r = ext_eval<V, Lanes32<V>>(d.ext + m.x, m.w & 31u, m.y, [&](uint32_t ref) {
    return ldr32<V>(s.state, ref, s.n_pad, lane);
  });
  const uint32_t mk = wmask32(ctl_width(m.w));
#pragma unroll
  for (int v = 0; v < V; v++) r.x[v] &= mk;
  return r;
}

// Activity of V consecutive lanes as a bit mask (bit v = lane + v active).
template <int V>
__device__ __forceinline__ uint32_t act_mask(const DSim& s, uint32_t lane, uint32_t cyc) {
  uint32_t m = 0;
#pragma unroll
  for (int v = 0; v < V; v++)
    if (lane_active(s, lane + v, cyc)) m |= 1u << v;
  return m;
}

// Store the active lanes (mask bit v = lane + v) of a result into a row;
// frozen instances keep their state.  Values already fit the row's class.
template <int V>
__device__ __forceinline__ void str(uint8_t* st, uint32_t ref, size_t np, uint32_t lane,
                                    const Lanes<V>& r, uint32_t m) {
  if constexpr (V == 2) {
    if (m == 3u) {
      uint8_t* p = const_cast<uint8_t*>(elem(st, ref, np, lane));
      switch (ref >> 30) {
        case 0: *reinterpret_cast<uint16_t*>(p) = (uint16_t)(r.x[0] | (r.x[1] << 8)); break;
        case 1: *reinterpret_cast<uint32_t*>(p) = (uint32_t)(r.x[0] | (r.x[1] << 16)); break;
        case 2: *reinterpret_cast<uint2*>(p) = make_uint2((uint32_t)r.x[0], (uint32_t)r.x[1]); break;
        default: *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(r.x[0], r.x[1]); break;
      }
      return;
    }
  } else if constexpr (V == 4) {
    if (m == 15u) {
      uint8_t* p = const_cast<uint8_t*>(elem(st, ref, np, lane));
      switch (ref >> 30) {
        case 0:
          *reinterpret_cast<uint32_t*>(p) =
              (uint32_t)(r.x[0] | (r.x[1] << 8) | (r.x[2] << 16) | (r.x[3] << 24));
          break;
        case 1:
          *reinterpret_cast<uint2*>(p) = make_uint2((uint32_t)(r.x[0] | (r.x[1] << 16)),
                                                    (uint32_t)(r.x[2] | (r.x[3] << 16)));
          break;
        case 2:
          *reinterpret_cast<uint4*>(p) = make_uint4((uint32_t)r.x[0], (uint32_t)r.x[1],
                                                    (uint32_t)r.x[2], (uint32_t)r.x[3]);
          break;
        default:
          reinterpret_cast<ulonglong2*>(p)[0] = make_ulonglong2(r.x[0], r.x[1]);
          reinterpret_cast<ulonglong2*>(p)[1] = make_ulonglong2(r.x[2], r.x[3]);
          break;
      }
      return;
    }
  } else if constexpr (V == 8) {
    if (m == 255u) {
      uint8_t* p = const_cast<uint8_t*>(elem(st, ref, np, lane));
      switch (ref >> 30) {
        case 0: {
          uint32_t lo = 0, hi = 0;
#pragma unroll
          for (int v = 0; v < 4; v++) {
            lo |= (uint32_t)r.x[v] << (8 * v);
            hi |= (uint32_t)r.x[4 + v] << (8 * v);
          }
          *reinterpret_cast<uint2*>(p) = make_uint2(lo, hi);
        } break;
        case 1:
          *reinterpret_cast<uint4*>(p) =
              make_uint4((uint32_t)(r.x[0] | (r.x[1] << 16)), (uint32_t)(r.x[2] | (r.x[3] << 16)),
                         (uint32_t)(r.x[4] | (r.x[5] << 16)), (uint32_t)(r.x[6] | (r.x[7] << 16)));
          break;
        case 2:
          reinterpret_cast<uint4*>(p)[0] =
              make_uint4((uint32_t)r.x[0], (uint32_t)r.x[1], (uint32_t)r.x[2], (uint32_t)r.x[3]);
          reinterpret_cast<uint4*>(p)[1] =
              make_uint4((uint32_t)r.x[4], (uint32_t)r.x[5], (uint32_t)r.x[6], (uint32_t)r.x[7]);
          break;
        default:
#pragma unroll
          for (int q = 0; q < 4; q++)
            reinterpret_cast<ulonglong2*>(p)[q] = make_ulonglong2(r.x[2 * q], r.x[2 * q + 1]);
          break;
      }
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < V; v++)
    if (m & (1u << v)) st1(st, ref, np, lane + v, r.x[v]);
}

// ---- packed byte lanes (SIMD within a register).  A narrow op whose result
// row is of class 0 (at most 8 bits) is evaluated for its V = 4 or 8 lanes as
// one word of V bytes: class-0 operand rows are used as they are loaded, the
// result is stored as it is computed, and no lane is unpacked.  That is exact
// when every operand row is of class 0 (each byte is a whole value), and for
// the ops whose low 8 result bits depend only on the operands' low 8 bits --
// the bitwise ops, add, subtract, shift left, cat and mux (a mux's selector is
// bit 0) -- whatever the operands' classes: wider operand rows are then cut to
// their low bytes as they are loaded.  Multiply and the dynamic shifts, and
// the ops that read whole operand values (right shifts, bit extraction,
// compares, reductions) on wider operand rows, keep the lane-by-lane form.
constexpr uint32_t PACK_LOW_OPS = (1u << OP_COPY) | (1u << OP_AND) | (1u << OP_OR) | (1u << OP_XOR) |
                                  (1u << OP_NOT) | (1u << OP_ADD) | (1u << OP_SUB) | (1u << OP_SHL) |
                                  (1u << OP_CAT) | (1u << OP_MUX);
constexpr uint32_t PACK_BYTE_OPS = (1u << OP_SHR) | (1u << OP_BITS) | (1u << OP_EQ) | (1u << OP_NEQ) |
                                   (1u << OP_LT) | (1u << OP_LEQ) | (1u << OP_GT) | (1u << OP_GEQ) |
                                   (1u << OP_ANDR) | (1u << OP_ORR) | (1u << OP_XORR);

// Whether a narrow op (descriptor m, result row dref) takes the packed form.
__device__ __forceinline__ bool packable(const uint4& m, uint32_t dref) {
  const uint32_t op = m.w & 31u;
  const bool bytes_in = ((m.x | m.y | m.z) >> 30) == 0u;  // every operand row of class 0
  return (dref >> 30) == 0u && (((PACK_LOW_OPS >> op) & 1u) || (bytes_in && ((PACK_BYTE_OPS >> op) & 1u)));
}

template <int V>
struct Packed;
template <>
struct Packed<4> {
  using T = uint32_t;
};
template <>
struct Packed<8> {
  using T = uint64_t;
};

// byte b in every byte of a packed word
template <typename T>
__device__ __forceinline__ T rep8(uint32_t b) {
  return (T)0x0101010101010101ull * (T)(b & 0xFFu);
}

// low byte of each of four 32-bit words
__device__ __forceinline__ uint32_t low_bytes4(uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  return __byte_perm(__byte_perm(x, y, 0x0040u), __byte_perm(z, w, 0x0040u), 0x5410u);
}

// V lanes of a row as V bytes: a class-0 row as stored, a class-1 or class-2
// row cut to the low byte of every lane.
template <int V>
__device__ __forceinline__ typename Packed<V>::T ldp(const uint8_t* st, uint32_t ref, size_t np, uint32_t lane) {
  const uint8_t* p = elem(st, ref, np, lane);
  const uint32_t k = ref >> 30;
  if constexpr (V == 8) {
    if (k == 0) {
      const uint2 t = *reinterpret_cast<const uint2*>(p);
      return (uint64_t)t.x | ((uint64_t)t.y << 32);
    }
    if (k == 1) {
      const uint4 t = *reinterpret_cast<const uint4*>(p);
      return (uint64_t)__byte_perm(t.x, t.y, 0x6420u) | ((uint64_t)__byte_perm(t.z, t.w, 0x6420u) << 32);
    }
    const uint4 t0 = reinterpret_cast<const uint4*>(p)[0];
    const uint4 t1 = reinterpret_cast<const uint4*>(p)[1];
    return (uint64_t)low_bytes4(t0.x, t0.y, t0.z, t0.w) | ((uint64_t)low_bytes4(t1.x, t1.y, t1.z, t1.w) << 32);
  } else {
    if (k == 0) return *reinterpret_cast<const uint32_t*>(p);
    if (k == 1) {
      const uint2 t = *reinterpret_cast<const uint2*>(p);
      return __byte_perm(t.x, t.y, 0x6420u);
    }
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    return low_bytes4(t.x, t.y, t.z, t.w);
  }
}

// Per byte: bit 7 set where the byte is not zero.
template <typename T>
__device__ __forceinline__ T nonzero8(T x) {
  const T L7 = rep8<T>(0x7Fu);
  return (((x & L7) + L7) | x) & rep8<T>(0x80u);
}

// Per byte: bit 7 set where a < b (unsigned).  (a | 0x80) - (b & 0x7F) keeps
// every byte's difference in 1..255 (no borrow between bytes); its bit 7 says
// whether a's low seven bits are at least b's.  Where the top bits of a and b
// differ, a < b exactly when b's is set.
template <typename T>
__device__ __forceinline__ T ltu8(T a, T b) {
  const T H = rep8<T>(0x80u);
  const T d = (a | H) - (b & ~H);
  const T x = a ^ b;
  return ((x & b) | (~x & ~d)) & H;
}

// Per byte: a + b and a - b mod 256 (the seven low bits added or subtracted
// without crossing into the next byte, the top bit fixed up by parity).
template <typename T>
__device__ __forceinline__ T add8(T a, T b) {
  const T H = rep8<T>(0x80u);
  return ((a & ~H) + (b & ~H)) ^ ((a ^ b) & H);
}
template <typename T>
__device__ __forceinline__ T sub8(T a, T b) {
  const T H = rep8<T>(0x80u);
  return ((a | H) - (b & ~H)) ^ ((a ^ ~b) & H);
}

// Per byte: a << s and a >> s (s < 8), the bits that cross a byte boundary removed.
template <typename T>
__device__ __forceinline__ T shl8(T a, uint32_t s) {
  return s >= 8u ? (T)0 : (a << s) & rep8<T>(0xFFu << s);
}
template <typename T>
__device__ __forceinline__ T shr8(T a, uint32_t s) {
  return s >= 8u ? (T)0 : (a >> s) & rep8<T>(0xFFu >> s);
}

// The op (ctl) on packed operand bytes a, b, c; the result masked to its width
// (at most 8 bits).  Follows the definitions of alu32_v lane by lane.
template <typename T>
__device__ __forceinline__ T alu_packed(uint32_t ctl, T a, T b, T c) {
  const uint32_t op = ctl & 31u, ar = (ctl >> 5) & 3u;
  const uint32_t p0 = (ctl >> 16) & 255u, p1 = ctl >> 24;
  const T ONE = rep8<T>(1u);
  T r;
  switch (op) {
    case OP_COPY: r = a; break;
    case OP_AND: r = a & b; if (ar == 3) r &= c; break;
    case OP_OR: r = a | b; if (ar == 3) r |= c; break;
    case OP_XOR: r = a ^ b; if (ar == 3) r ^= c; break;
    case OP_NOT: r = ~a; break;
    case OP_ADD: r = add8(a, b); if (ar == 3) r = add8(r, c); break;
    case OP_SUB: r = sub8(a, b); break;
    case OP_SHL: r = shl8(a, p0); break;
    case OP_SHR: r = shr8(a, p0); break;
    case OP_BITS: r = shr8(a, p1) & rep8<T>(wmask32(p0 - p1 + 1u)); break;
    case OP_CAT: r = shl8(a, p0) | b; break;
    case OP_EQ: r = (nonzero8(a ^ b) >> 7) ^ ONE; break;
    case OP_NEQ: r = nonzero8(a ^ b) >> 7; break;
    case OP_LT: r = ltu8(a, b) >> 7; break;
    case OP_LEQ: r = (ltu8(b, a) >> 7) ^ ONE; break;
    case OP_GT: r = ltu8(b, a) >> 7; break;
    case OP_GEQ: r = (ltu8(a, b) >> 7) ^ ONE; break;
    case OP_MUX: {
      const T s = (a & ONE) * (T)0xFFu;  // 0xFF where the selector bit is set
      r = (b & s) | (c & ~s);
    } break;
    case OP_ANDR: {  // all of the low p0 bits set (none can be above bit 7)
      const T mm = rep8<T>(wmask32(p0));
      r = p0 > 8u ? (T)0 : (nonzero8((a & mm) ^ mm) >> 7) ^ ONE;
    } break;
    case OP_ORR: r = nonzero8(a) >> 7; break;
    case OP_XORR: {
      T x = a ^ (a >> 4);  // bit 0 of each byte folds in its own bits only
      x ^= x >> 2;
      x ^= x >> 1;
      r = x & ONE;
    } break;
    default: r = 0; break;
  }
  return r & rep8<T>(0xFFu >> (8u - ctl_width(ctl)));
}

// Store the active lanes (mask bit v = lane + v) of a packed class-0 result.
template <int V>
__device__ __forceinline__ void stp(uint8_t* st, uint32_t ref, size_t np, uint32_t lane,
                                    typename Packed<V>::T r, uint32_t m) {
  uint8_t* p = const_cast<uint8_t*>(elem(st, ref, np, lane));
  if (m == (1u << V) - 1u) {
    if constexpr (V == 8)
      *reinterpret_cast<uint2*>(p) = make_uint2((uint32_t)r, (uint32_t)(r >> 32));
    else
      *reinterpret_cast<uint32_t*>(p) = r;
    return;
  }
#pragma unroll
  for (int v = 0; v < V; v++)
    if (m & (1u << v)) p[v] = (uint8_t)(r >> (8 * v));
}

// One packed item: every operand load issued before the evaluation.
template <int V>
__device__ __forceinline__ void item_packed(uint8_t* st, size_t np, uint32_t lane, const uint4& m,
                                            uint32_t dref, uint32_t am) {
  using T = typename Packed<V>::T;
  const uint32_t ar = (m.w >> 5) & 3u;
  const T a = ldp<V>(st, m.x, np, lane);
  const T b = ar >= 2 ? ldp<V>(st, m.y, np, lane) : (T)0;
  const T c = ar >= 3 ? ldp<V>(st, m.z, np, lane) : (T)0;
  stp<V>(st, dref, np, lane, alu_packed<T>(m.w, a, b, c), am);
}

// One narrow item: gather, evaluate, store.
template <int V>
__device__ __forceinline__ void item32(uint8_t* st, size_t np, uint32_t lane, const uint4& m,
                                       uint32_t dref, uint32_t am) {
  if constexpr (V == 4 || V == 8) {
    if (packable(m, dref)) {
      item_packed<V>(st, np, lane, m, dref, am);
      return;
    }
  }
  Lanes32<V> a, b, c;
  const uint32_t ar = (m.w >> 5) & 3u;
  a = ldr32<V>(st, m.x, np, lane);
#pragma unroll
  for (int v = 0; v < V; v++) b.x[v] = c.x[v] = 0u;
  if (ar >= 2) b = ldr32<V>(st, m.y, np, lane);
  if (ar >= 3) c = ldr32<V>(st, m.z, np, lane);
  str32<V>(st, dref, np, lane, alu32_v<V>(m.w, a, b, c), am);
}

// Operand gather of one op with at most three operands for V lanes
// (OI = LI . OIM for this s coordinate).
template <int V>
__device__ __forceinline__ void gather(const uint8_t* st, size_t np, uint32_t lane, const uint4& m,
                                       Lanes<V>& a, Lanes<V>& b, Lanes<V>& c) {
#pragma unroll
  for (int v = 0; v < V; v++) a.x[v] = b.x[v] = c.x[v] = 0;
  const uint32_t ar = (m.w >> 5) & 3u;
  a = ldr<V>(st, m.x, np, lane);
  if (ar >= 2) b = ldr<V>(st, m.y, np, lane);
  if (ar >= 3) c = ldr<V>(st, m.z, np, lane);
}

// op_u / op_r / op_s of one op with at most three operands for V lanes, from
// gathered operands.
template <int V>
__device__ __forceinline__ Lanes<V> apply(const DDesign& d, const DSim& s, const uint4& m,
                                          const Lanes<V>& a, const Lanes<V>& b, const Lanes<V>& c,
                                          uint32_t lane) {
  const uint32_t ctl = m.w;
  Lanes<V> r;
  if ((ctl & 31u) == OP_MEMRD) {
#pragma unroll
    for (int v = 0; v < V; v++) r.x[v] = eval_memrd(d, s, ctl, a.x[v], lane + v);
  } else {
    r = alu_v<V>(ctl, a, b, c);
  }
  return r;
}

// Row kinds of a layer, in their order: narrow (<= 3 operands), wide (<= 3
// operands), extended (> 3 operands in the side array).
enum : int { ROW_NARROW = 0, ROW_WIDE = 1, ROW_EXT = 2 };

template <int V, int KIND>
__device__ __forceinline__ void item_of_kind(const DDesign& d, const DSim& s, uint32_t lane, const uint4& m,
                                             uint32_t dref, uint32_t am) {
  if constexpr (KIND == ROW_NARROW) {
    item32<V>(s.state, s.n_pad, lane, m, dref, am);
  } else if constexpr (KIND == ROW_WIDE) {
    Lanes<V> va, vb, vc;
    gather<V>(s.state, s.n_pad, lane, m, va, vb, vc);
    str<V>(s.state, dref, s.n_pad, lane, apply<V>(d, s, m, va, vb, vc, lane), am);
  } else {
    if (m.w & CTL_NARROW)
      str32<V>(s.state, dref, s.n_pad, lane, eval_ext32_v<V>(d, s, m, lane), am);
    else
      str<V>(s.state, dref, s.n_pad, lane, eval_ext_v<V>(d, s, m, lane), am);
  }
}

// This thread's rows r, r + stride, ... below r_end of one kind (fixed lane
// chunk), descriptors read from global memory one row ahead; returns the
// thread's first row at or past r_end (where the next kind continues).
template <int V, int KIND>
__device__ __forceinline__ uint32_t walk_rows(const DDesign& d, const DSim& s, uint32_t op0, uint32_t r,
                                              uint32_t r_end, uint32_t stride, uint32_t lane, uint32_t am) {
  if (r >= r_end) return r;
  uint4 m = __ldg(&d.meta[op0 + r]);
  uint32_t dref = __ldg(&d.dst[op0 + r]);
  for (;;) {
    const uint32_t rn = r + stride;
    uint4 mn = make_uint4(0, 0, 0, 0);
    uint32_t dn = 0;
    if (rn < r_end) {
      mn = __ldg(&d.meta[op0 + rn]);
      dn = __ldg(&d.dst[op0 + rn]);
    }
    item_of_kind<V, KIND>(d, s, lane, m, dref, am);
    if (rn >= r_end) return rn;
    r = rn;
    m = mn;
    dref = dn;
  }
}

// The same with U rows in flight per thread: the U rows' descriptors, then
// all their operand gathers, then their results (more memory-level
// parallelism per thread at the price of registers; 64-bit lanes throughout).
template <int V, int KIND, int U>
__device__ __forceinline__ uint32_t walk_rows_u(const DDesign& d, const DSim& s, uint32_t op0, uint32_t r,
                                                uint32_t r_end, uint32_t stride, uint32_t lane, uint32_t am) {
  if constexpr (U == 1 || KIND == ROW_EXT) {
    return walk_rows<V, KIND>(d, s, op0, r, r_end, stride, lane, am);
  } else {
    if (r >= r_end) return r;
    // the thread's first row at or past r_end: the next kind starts there
    const uint32_t next = r + (r_end - r + stride - 1u) / stride * stride;
    for (; r < r_end; r += U * stride) {
      uint4 m[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        ok[u] = r + u * stride < r_end;
        m[u] = ok[u] ? __ldg(&d.meta[op0 + r + u * stride]) : make_uint4(0, 0, 0, 0);
      }
      Lanes<V> va[U], vb[U], vc[U];
#pragma unroll
      for (int u = 0; u < U; u++)
        if (ok[u]) gather<V>(s.state, s.n_pad, lane, m[u], va[u], vb[u], vc[u]);
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (!ok[u]) continue;
        const Lanes<V> res = apply<V>(d, s, m[u], va[u], vb[u], vc[u], lane);
        str<V>(s.state, __ldg(&d.dst[op0 + r + u * stride]), s.n_pad, lane, res, am);
      }
    }
    return next;
  }
}

// Generic mapping (more lane chunks than threads): kept out of line so that it
// does not cost the fixed-mapping hot loop any registers.
template <int V, int U>
__device__ __noinline__ void eval_ops_generic(const DDesign& d, const DSim& s, uint32_t op0,
                                              uint32_t n_rows, const ItemSpace& is, uint32_t cyc) {
  const size_t np = s.n_pad;
  const uint32_t n_items = n_rows * is.tpo.d;
  for (uint32_t i0 = is.first; i0 < n_items; i0 += is.stride * U) {
    uint4 m[U];
    uint32_t row[U], lane[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint32_t i = i0 + u * is.stride;
      ok[u] = i < n_items;
      row[u] = fdiv(is.tpo, i);
      lane[u] = is.lane_base + (i - row[u] * is.tpo.d) * V;
      m[u] = ok[u] ? __ldg(&d.meta[op0 + row[u]]) : make_uint4(0, 0, 0, 0);
    }
    Lanes<V> va[U], vb[U], vc[U];
#pragma unroll
    for (int u = 0; u < U; u++)
      if (ok[u]) gather<V>(s.state, np, lane[u], m[u], va[u], vb[u], vc[u]);
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (!ok[u]) continue;
      const Lanes<V> res = apply<V>(d, s, m[u], va[u], vb[u], vc[u], lane[u]);
      str<V>(s.state, __ldg(&d.dst[op0 + row[u]]), np, lane[u], res, act_mask<V>(s, lane[u], cyc));
    }
  }
}


// (a2) evaluate ops [op0, op0 + n_rows) of the lowered list, none of them with
// more than three operands.  U ops are issued
// per thread before any result is stored, so all their operand loads are in
// flight together (memory-level parallelism).
template <int V, int U>
__device__ __forceinline__ void eval_ops(const DDesign& d, const DSim& s, uint32_t op0,
                                         uint32_t n_rows, const ItemSpace& is, uint32_t cyc) {
  const size_t np = s.n_pad;
  if (!is.row_stride) {
    eval_ops_generic<V, U>(d, s, op0, n_rows, is, cyc);
    return;
  }
  {
    if (is.row0 == NO_ROW) return;
    const uint32_t am = act_mask<V>(s, is.lane, cyc);
    if (!am) return;
    const uint4* meta = d.meta + op0;
    const uint32_t* dst = d.dst + op0;
    if constexpr (U == 1) {
      // descriptor of the next row fetched one step ahead: the dependent chain of
      // an item is then operand loads -> compute -> store
      uint32_t r = is.row0;
      if (r >= n_rows) return;
      uint4 m = __ldg(&meta[r]);
      uint32_t dref = __ldg(&dst[r]);
      for (;;) {
        const uint32_t rn = r + is.row_stride;
        uint4 mn = make_uint4(0, 0, 0, 0);
        uint32_t dn = 0;
        if (rn < n_rows) {
          mn = __ldg(&meta[rn]);
          dn = __ldg(&dst[rn]);
        }
        if (m.w & CTL_NARROW) {
          item32<V>(s.state, np, is.lane, m, dref, am);
        } else {
          Lanes<V> va, vb, vc;
          gather<V>(s.state, np, is.lane, m, va, vb, vc);
          const Lanes<V> res = apply<V>(d, s, m, va, vb, vc, is.lane);
          str<V>(s.state, dref, np, is.lane, res, am);
        }
        if (rn >= n_rows) break;
        r = rn;
        m = mn;
        dref = dn;
      }
      return;
    }
    for (uint32_t r0 = is.row0; r0 < n_rows; r0 += is.row_stride * U) {
      uint4 m[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint32_t r = r0 + u * is.row_stride;
        ok[u] = r < n_rows;
        m[u] = ok[u] ? __ldg(&meta[r]) : make_uint4(0, 0, 0, 0);
      }
      Lanes<V> va[U], vb[U], vc[U];
#pragma unroll
      for (int u = 0; u < U; u++)
        if (ok[u]) gather<V>(s.state, np, is.lane, m[u], va[u], vb[u], vc[u]);
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (!ok[u]) continue;
        const Lanes<V> res = apply<V>(d, s, m[u], va[u], vb[u], vc[u], is.lane);
        str<V>(s.state, __ldg(&dst[r0 + u * is.row_stride]), np, is.lane, res, am);
      }
    }
  }
}

// Visit (row, first lane) pairs of n_rows rows under either mapping.
template <int V, typename F>
__device__ __forceinline__ void for_rows(const ItemSpace& is, uint32_t n_rows, F&& f) {
  if (is.row_stride) {
    if (is.row0 == NO_ROW) return;
    for (uint32_t r = is.row0; r < n_rows; r += is.row_stride) f(r, is.lane);
  } else {
    const uint32_t n_items = n_rows * is.tpo.d;
    for (uint32_t i = is.first; i < n_items; i += is.stride) {
      const uint32_t r = fdiv(is.tpo, i);
      f(r, is.lane_base + (i - r * is.tpo.d) * V);
    }
  }
}

// Ops [op0, op0 + n_rows) with more than three operands (fused mux chains,
// wide folds), after the layer's common loop.
template <int V>
__device__ __forceinline__ void eval_ext_rows(const DDesign& d, const DSim& s, uint32_t op0,
                                           uint32_t n_rows, const ItemSpace& is, uint32_t cyc) {
  if (is.row_stride) {  // fixed lane chunk: activity once, descriptor one row ahead
    if (is.row0 == NO_ROW || is.row0 >= n_rows) return;
    const uint32_t am = act_mask<V>(s, is.lane, cyc);
    if (!am) return;
    uint32_t r = is.row0;
    uint4 m = __ldg(&d.meta[op0 + r]);
    for (;;) {
      const uint32_t rn = r + is.row_stride;
      const uint4 mn = rn < n_rows ? __ldg(&d.meta[op0 + rn]) : m;
      const uint32_t dref = __ldg(&d.dst[op0 + r]);
      if (m.w & CTL_NARROW)
        str32<V>(s.state, dref, s.n_pad, is.lane, eval_ext32_v<V>(d, s, m, is.lane), am);
      else
        str<V>(s.state, dref, s.n_pad, is.lane, eval_ext_v<V>(d, s, m, is.lane), am);
      if (rn >= n_rows) break;
      r = rn;
      m = mn;
    }
    return;
  }
  for_rows<V>(is, n_rows, [&](uint32_t r, uint32_t lane) {
    const uint32_t am = act_mask<V>(s, lane, cyc);
    if (!am) return;
    const Lanes<V> res = eval_ext_v<V>(d, s, __ldg(&d.meta[op0 + r]), lane);
    str<V>(s.state, __ldg(&d.dst[op0 + r]), s.n_pad, lane, res, am);
  });
}

// (a2) one layer: its ops with at most three operands, then the others, in
// one phase (no dependence inside a layer).
template <int V, int U>
__device__ __forceinline__ void eval_layer(const DDesign& d, const DSim& s, uint32_t L,
                                           const ItemSpace& is, uint32_t cyc) {
  const uint32_t o0 = __ldg(&d.layer_off[L]), e = __ldg(&d.layer_ext[L]);
  const uint32_t o1 = __ldg(&d.layer_off[L + 1]);
  if (!is.row_stride) {  // generic mapping
    eval_ops<V, U>(d, s, o0, e - o0, is, cyc);
    if (e < o1) eval_ext_rows<V>(d, s, e, o1 - e, is, cyc);
    return;
  }
  // fixed lane chunk: one row sequence over the layer, kind by kind
  if (is.row0 == NO_ROW || is.row0 >= o1 - o0) return;
  const uint32_t am = act_mask<V>(s, is.lane, cyc);
  if (!am) return;
  const uint32_t nw = __ldg(&d.layer_wide[L]) - o0;
  uint32_t r = walk_rows_u<V, ROW_NARROW, U>(d, s, o0, is.row0, nw, is.row_stride, is.lane, am);
  r = walk_rows_u<V, ROW_WIDE, U>(d, s, o0, r, e - o0, is.row_stride, is.lane, am);
  walk_rows<V, ROW_EXT>(d, s, o0, r, o1 - o0, is.row_stride, is.lane, am);
}

// ---- activity-aware evaluation (the cascade-level "skip what did not change"
// optimisation): an op is evaluated for a 128-lane chunk only if one of its
// operand rows changed in that chunk during this cycle (stamp == cycle), and
// its result is written and stamped only if it differs from the stored value.
// Skipping is exact: an op whose operands are unchanged has an unchanged
// result.  Stamps are 8-bit, so a stamp 256 cycles old reads as current --
// that only evaluates an op again (no change, no stamp), never skips one.
// Requires the fixed lane mapping (the launch guarantees it).
template <int V>
__device__ __forceinline__ bool any_diff(const Lanes<V>& a, const Lanes<V>& b, uint32_t am) {
  bool d = false;
#pragma unroll
  for (int v = 0; v < V; v++) d |= ((am >> v) & 1u) && a.x[v] != b.x[v];
  return d;
}

template <int V>
__device__ __forceinline__ bool any_diff32(const Lanes32<V>& a, const Lanes32<V>& b, uint32_t am) {
  bool d = false;
#pragma unroll
  for (int v = 0; v < V; v++) d |= ((am >> v) & 1u) && a.x[v] != b.x[v];
  return d;
}

// Is row r hot for lane chunks [ch_lo, ch_hi]: an operand stamped this cycle?
__device__ __forceinline__ bool row_hot(const DDesign& d, const DSim& s, const uint4& m, bool ext, uint32_t ch_lo,
                                        uint32_t ch_hi, uint8_t g) {
  if ((m.w & 31u) == OP_MEMRD) return true;  // memory contents carry no stamps
  auto hot_ref = [&](uint32_t ref) {
    const uint8_t* a = s.act + (size_t)row_index(d, ref) * s.act_chunks;
    bool h = a[ch_lo] == g;
    if (ch_hi != ch_lo) h |= a[ch_hi] == g;
    return h;
  };
  if (ext) {
    const uint32_t* a = d.ext + m.x;
    for (uint32_t i = 0; i < m.y; i++)
      if (hot_ref(__ldg(&a[i]))) return true;
    return false;
  }
  const uint32_t ar = (m.w >> 5) & 3u;
  bool h = hot_ref(m.x);
  if (ar >= 2) h |= hot_ref(m.y);
  if (ar >= 3) h |= hot_ref(m.z);
  return h;
}

// Evaluate one hot row for this thread's V lanes; store and stamp on change.
template <int V>
__device__ __forceinline__ void act_item(const DDesign& d, const DSim& s, const uint4& m, uint32_t dref, bool ext,
                                         uint32_t lane, uint32_t am, uint8_t g) {
  const size_t np = s.n_pad;
  bool changed;
  if (m.w & CTL_NARROW) {
    Lanes32<V> res;
    if (ext) {
      res = eval_ext32_v<V>(d, s, m, lane);
    } else {
      Lanes32<V> a, b, c;
      const uint32_t ar = (m.w >> 5) & 3u;
      a = ldr32<V>(s.state, m.x, np, lane);
#pragma unroll
      for (int v = 0; v < V; v++) b.x[v] = c.x[v] = 0u;
      if (ar >= 2) b = ldr32<V>(s.state, m.y, np, lane);
      if (ar >= 3) c = ldr32<V>(s.state, m.z, np, lane);
      res = alu32_v<V>(m.w, a, b, c);
    }
    changed = any_diff32<V>(res, ldr32<V>(s.state, dref, np, lane), am);
    if (changed) str32<V>(s.state, dref, np, lane, res, am);
  } else {
    Lanes<V> res;
    if (ext) {
      res = eval_ext_v<V>(d, s, m, lane);
    } else {
      Lanes<V> va, vb, vc;
      gather<V>(s.state, np, lane, m, va, vb, vc);
      res = apply<V>(d, s, m, va, vb, vc, lane);
    }
    changed = any_diff<V>(res, ldr<V>(s.state, dref, np, lane), am);
    if (changed) str<V>(s.state, dref, np, lane, res, am);
  }
  if (changed) *act_at(d, s, dref, lane) = g;
}

template <int V>
__device__ __forceinline__ void eval_ops_act(const DDesign& d, const DSim& s, uint32_t op0, uint32_t n_rows,
                                             uint32_t n_plain, const ItemSpace& is, uint32_t cyc,
                                             uint32_t& n_eval, uint32_t& n_skip) {
  if (is.row0 == NO_ROW) return;
  const uint32_t am = act_mask<V>(s, is.lane, cyc);
  const uint8_t g = (uint8_t)(s.act_g0 + cyc);
  const bool force = s.act_force && cyc == 0;
  if (is.tpo.d % 32u == 0u) {
    // Warp-cooperative: the warp's 32 threads share one row sequence and one
    // lane range, so lane i checks row (base + i) of that sequence, a ballot
    // collects the hot ones, and the whole warp evaluates only those -- one
    // round of descriptor and stamp loads per 32 rows.
    const uint32_t lid = threadIdx.x & 31u;
    const uint32_t first = is.lane - lid * V;
    const uint32_t ch_lo = first >> 7, ch_hi = (first + 32u * V - 1u) >> 7;
    const bool warp_idle = __ballot_sync(0xFFFFFFFFu, am != 0u) == 0u;
    if (warp_idle) return;
    for (uint32_t base = 0;; base += 32u) {
      const uint32_t r = is.row0 + (base + lid) * is.row_stride;
      const bool valid = r < n_rows;
      uint4 m = make_uint4(0, 0, 0, 0);
      bool hot = false;
      if (valid) {
        m = __ldg(&d.meta[op0 + r]);
        hot = force || row_hot(d, s, m, r >= n_plain, ch_lo, ch_hi, g);
      }
      uint32_t hm = __ballot_sync(0xFFFFFFFFu, hot);
      const uint32_t vm = __ballot_sync(0xFFFFFFFFu, valid);
      if (am) {
        n_eval += __popc(hm);
        n_skip += __popc(vm) - __popc(hm);
      }
      while (hm) {
        const uint32_t k = __ffs(hm) - 1u;
        hm &= hm - 1u;
        uint4 mk;
        mk.x = __shfl_sync(0xFFFFFFFFu, m.x, k);
        mk.y = __shfl_sync(0xFFFFFFFFu, m.y, k);
        mk.z = __shfl_sync(0xFFFFFFFFu, m.z, k);
        mk.w = __shfl_sync(0xFFFFFFFFu, m.w, k);
        const uint32_t rk = is.row0 + (base + k) * is.row_stride;
        if (am) act_item<V>(d, s, mk, __ldg(&d.dst[op0 + rk]), rk >= n_plain, is.lane, am, g);
      }
      if (vm != 0xFFFFFFFFu) break;  // the sequence ended inside this round
    }
    return;
  }
  // one thread, one row at a time (lane ranges narrower than a warp)
  if (!am) return;
  for (uint32_t r = is.row0; r < n_rows; r += is.row_stride) {
    const uint4 m = __ldg(&d.meta[op0 + r]);
    const bool ext = r >= n_plain;
    if (!(force || row_hot(d, s, m, ext, is.lane >> 7, is.lane >> 7, g))) {
      n_skip++;
      continue;
    }
    n_eval++;
    act_item<V>(d, s, m, __ldg(&d.dst[op0 + r]), ext, is.lane, am, g);
  }
}

template <int V>
__device__ __forceinline__ void eval_layer_act(const DDesign& d, const DSim& s, uint32_t L, const ItemSpace& is,
                                               uint32_t cyc, uint32_t& n_eval, uint32_t& n_skip) {
  const uint32_t o0 = __ldg(&d.layer_off[L]), e = __ldg(&d.layer_ext[L]);
  const uint32_t o1 = __ldg(&d.layer_off[L + 1]);
  eval_ops_act<V>(d, s, o0, o1 - o0, e - o0, is, cyc, n_eval, n_skip);
}

// (a1) primary inputs for cycle cyc.
template <int V>
__device__ __forceinline__ void stim_items(const DDesign& d, const DSim& s, const ItemSpace& is,
                                           uint32_t cyc) {
  if (s.stim_mode == 0) return;
  const size_t np = s.n_pad;
  for_rows<V>(is, d.n_inputs, [&](uint32_t j, uint32_t lane0) {
    const uint64_t mk = wmask(__ldg(&d.in_w[j]));
#pragma unroll
    for (int v = 0; v < V; v++) {
      const uint32_t lane = lane0 + v;
      if (!lane_active(s, lane, cyc)) continue;
      uint64_t x;
      if (s.stim_mode == 1) {  // xorshift64 (Marsaglia 2003), shifts 13, 7, 17
        x = s.xs[(size_t)j * np + lane];
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        s.xs[(size_t)j * np + lane] = x;
      } else {
        x = __ldg(&s.stim[((size_t)cyc * d.n_inputs + j) * s.n_user + user_of(s, lane)]);
      }
      const uint32_t iref = __ldg(&d.in_ref[j]);
      if (s.act) {  // stamp only a change (held or repeated values cost nothing downstream)
        if (ld1(s.state, iref, np, lane) == (x & mk)) continue;
        *act_at(d, s, iref, lane) = (uint8_t)(s.act_g0 + cyc);
      }
      st1(s.state, iref, np, lane, x & mk);
    }
  });
}

// One register's clock edge for V lanes (D row dsrc, Q row qref, width mask mk):
// Q <- D, or the init value in reset cycles; with activity stamps, written
// only where it changes.
template <int V>
__device__ __forceinline__ void commit_reg(const DDesign& d, const DSim& s, uint32_t r, uint32_t lane, uint32_t cyc,
                                           uint32_t am, uint32_t dsrc, uint32_t qref, uint64_t mk) {
  const size_t np = s.n_pad;
  Lanes<V> v;
  if (s.reset) {
    const uint64_t init = __ldg(&d.reg_init[r]) & mk;
#pragma unroll
    for (int t = 0; t < V; t++) v.x[t] = init;
  } else {
    v = ldr<V>(s.state, dsrc, np, lane);
#pragma unroll
    for (int t = 0; t < V; t++) v.x[t] &= mk;
    if (s.reset_lane) {  // instances still in their leading reset cycles
      const uint64_t init = __ldg(&d.reg_init[r]) & mk;
#pragma unroll
      for (int t = 0; t < V; t++)
        if (cyc < __ldg(&s.reset_lane[lane + t])) v.x[t] = init;
    }
  }
  if (s.act) {  // write and stamp only what changes; visible from the next cycle
    const Lanes<V> q = ldr<V>(s.state, qref, np, lane);
    bool changed = false;
#pragma unroll
    for (int t = 0; t < V; t++) changed |= ((am >> t) & 1u) && q.x[t] != v.x[t];
    if (!changed) return;
    *act_at(d, s, qref, lane) = (uint8_t)(s.act_g0 + cyc + 1u);
  }
  str<V>(s.state, qref, np, lane, v, am);
}

// (a5) clock edge: registers (rows [0, n_regs)), then memory write ports
// (rows [n_regs, n_regs + n_mems), ports of one memory in port order).  In the
// fixed mapping a thread's registers are walked with the next register's
// table entries loaded one row ahead, so that an item's dependent chain is
// its D load and its store.
template <int V>
__device__ __forceinline__ void commit_items(const DDesign& d, const DSim& s, const ItemSpace& is,
                                             uint32_t cyc) {
  const size_t np = s.n_pad;
  uint32_t r0 = 0;  // first row for the generic walk below
  if (is.row_stride) {
    if (is.row0 == NO_ROW) return;
    const uint32_t am = act_mask<V>(s, is.lane, cyc);
    if (!am) return;
    uint32_t r = is.row0;
    if (r < d.n_regs) {
      uint32_t dsrc = __ldg(&d.reg_src[r]), qref = __ldg(&d.reg_ref[r]), w = __ldg(&d.reg_w[r]);
      for (;;) {
        const uint32_t rn = r + is.row_stride;
        uint32_t dn = 0, qn = 0, wn = 1;
        if (rn < d.n_regs) {
          dn = __ldg(&d.reg_src[rn]);
          qn = __ldg(&d.reg_ref[rn]);
          wn = __ldg(&d.reg_w[rn]);
        }
        commit_reg<V>(d, s, r, is.lane, cyc, am, dsrc, qref, wmask(w));
        r = rn;
        if (r >= d.n_regs) break;
        dsrc = dn;
        qref = qn;
        w = wn;
      }
    }
    r0 = r;  // the thread's first row past the registers: its memory ports
  }
  for_rows<V>(is, d.n_regs + d.n_mems, [&](uint32_t r, uint32_t lane) {
    if (r < r0 && is.row_stride) return;  // fixed mapping: registers done above
    const uint32_t am = act_mask<V>(s, lane, cyc);
    if (!am) return;
    if (r < d.n_regs) {
      commit_reg<V>(d, s, r, lane, cyc, am, __ldg(&d.reg_src[r]), __ldg(&d.reg_ref[r]), wmask(__ldg(&d.reg_w[r])));
    } else {
      const uint32_t mi = r - d.n_regs;
      const uint4 info = __ldg(&d.mem_info[mi]);
      const uint32_t p1 = __ldg(&d.mem_info[mi + 1]).w;
      const uint64_t mk = wmask(info.z);
#pragma unroll
      for (int t = 0; t < V; t++) {
        if (!(am & (1u << t))) continue;
        const uint32_t ln = lane + t;
        for (uint32_t p = info.w; p < p1; p++) {
          const uint4 w = __ldg(&d.wport[p]);
          if (ld1(s.state, w.y, np, ln) & 1ull) {
            const uint64_t a = ld1(s.state, w.z, np, ln) & (uint64_t)info.y;
            s.mem[((size_t)info.x + a) * np + ln] = ld1(s.state, w.w, np, ln) & mk;
          }
        }
      }
    }
  });
}

// (a7) per-cycle probes: end-of-cycle values of selected slots, or (waveform
// mode) one record per value change.
template <int V>
__device__ __forceinline__ void probe_items(const DSim& s, const ItemSpace& is, uint32_t cyc) {
  for_rows<V>(is, s.n_probe, [&](uint32_t p, uint32_t lane0) {
    const uint32_t slot = __ldg(&s.probe_slot[p]);
#pragma unroll
    for (int t = 0; t < V; t++) {
      const uint32_t lane = lane0 + t;
      if (!lane_active(s, lane, cyc)) continue;
      const uint64_t v = ld1(s.state, slot, s.n_pad, lane);
      if (s.probe_changes) {
        uint64_t* prev = s.probe_prev + (size_t)p * s.n_pad + lane;
        if (*prev != v) {
          *prev = v;
          const unsigned long long k = atomicAdd(s.change_count, 1ull);
          if (k < s.change_cap) {
            // 24-byte record {cycle, probe, instance, pad, value}: three 8-byte words
            // (records are only 8-byte aligned)
            uint64_t* rec = s.probe_out + 3 * k;
            rec[0] = (uint64_t)cyc | ((uint64_t)p << 32);
            rec[1] = (uint64_t)user_of(s, lane);
            rec[2] = v;
          }
        }
      } else {
        s.probe_out[((size_t)cyc * s.n_probe + p) * s.n_user + user_of(s, lane)] = v;
      }
    }
  });
}

}  // namespace rteaal
