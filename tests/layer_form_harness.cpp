// Test-only host harness for the LAYER and TILE forms: the library's own device functions
// (kernels.cuh: stim_items, eval_layer, commit_items) and lowering (lower.cpp),
// compiled with the host compiler, run phase by phase -- stimulus, every layer,
// clock edge -- with each phase called once per thread index.  Within a phase
// no item reads what another item writes (ops of one layer read lower layers
// only; the edge reads op rows and writes register rows), so running the
// thread indices one after another gives the result of any GPU interleaving.
// The CUDA built-ins those functions use are stood in for below; the warp
// votes and shuffles belong to activity-aware evaluation only, never used here.
#include <cuda_runtime.h>  // vector types (uint4, ...) and qualifiers for a host compile

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <map>
#include <mutex>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#ifndef __noinline__
#define __noinline__
#endif

static thread_local uint3 threadIdx;
static uint3 blockIdx, blockDim, gridDim;

// A warp of 32 host threads: ballots and shuffles exchange their values through
// one slot per lane between two barrier rounds.  Every caller reaches the same
// sequence of collectives (each branch that leads to one is warp-uniform).
struct Warp {
  std::atomic<unsigned> arrived{0}, generation{0};
  unsigned long long slot[32];
  void wait() {  // yields while waiting; a wait that never ends aborts instead of hanging
    const unsigned gen = generation.load();
    if (arrived.fetch_add(1) + 1 == 32) {
      arrived.store(0);
      generation.fetch_add(1);
      return;
    }
    for (unsigned long long spins = 0; generation.load() == gen; spins++) {
      if (spins > 2000000000ull) abort();
      std::this_thread::yield();
    }
  }
};
static thread_local Warp* warp = nullptr;

// The FLOW form's collectives: lanes of one warp (host threads) vote on a mask
// of the warp; each lane's n-th call with a given mask joins the n-th round of
// that mask, which ends once every lane of the mask has voted (lanes of the
// mask reach the same calls in the same order).  A round that does not fill
// within a minute aborts instead of hanging.
struct FlowWarp {
  std::mutex mu;
  std::condition_variable cv;
  struct Round {
    unsigned arrived = 0, left = 0, bits = 0;
  };
  std::map<std::pair<unsigned, unsigned>, Round> rounds;
  std::map<unsigned, unsigned> seq[32];
  unsigned vote(unsigned lane, unsigned mask, bool pred) {
    std::unique_lock<std::mutex> lk(mu);
    const auto key = std::make_pair(mask, seq[lane][mask]++);
    Round& r = rounds[key];
    if (pred) r.bits |= 1u << lane;
    const unsigned need = (unsigned)__builtin_popcount(mask);
    if (++r.arrived == need) {
      cv.notify_all();
    } else if (!cv.wait_for(lk, std::chrono::seconds(60), [&] { return r.arrived == need; })) {
      abort();
    }
    const unsigned bits = r.bits;
    if (++r.left == need) rounds.erase(key);
    return bits;
  }
};
static thread_local FlowWarp* flow_warp = nullptr;

template <typename T>
static inline T __ldg(const T* p) {
  return *p;
}
// byte n of the result = byte (selector nibble n & 7) of the 8-byte value {y, x}
static inline unsigned __byte_perm(unsigned x, unsigned y, unsigned s) {
  const unsigned long long v = ((unsigned long long)y << 32) | x;
  unsigned r = 0;
  for (int n = 0; n < 4; n++) r |= (unsigned)((v >> (8 * ((s >> (4 * n)) & 7u))) & 0xFFu) << (8 * n);
  return r;
}
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline int __popcll(unsigned long long x) { return __builtin_popcountll(x); }
static inline int __ffs(int x) { return __builtin_ffs(x); }
static inline unsigned __ballot_sync(unsigned mask, int pred) {
  if (flow_warp) return flow_warp->vote(threadIdx.x & 31u, mask, pred != 0);
  if (!warp) abort();
  const unsigned lid = threadIdx.x & 31u;
  warp->slot[lid] = pred ? 1u : 0u;
  warp->wait();
  unsigned r = 0;
  for (unsigned i = 0; i < 32; i++) r |= (unsigned)warp->slot[i] << i;
  warp->wait();
  return r;
}
template <typename T>
static inline T __shfl_sync(unsigned, T v, int src, int = 32) {
  if (!warp) abort();
  warp->slot[threadIdx.x & 31u] = (unsigned long long)v;
  warp->wait();
  const T r = (T)warp->slot[src & 31];
  warp->wait();
  return r;
}
static inline int __all_sync(unsigned mask, int pred) { return __ballot_sync(mask, pred) == mask; }
static inline int __any_sync(unsigned mask, int pred) { return __ballot_sync(mask, pred) != 0u; }
static inline unsigned atomicOr(unsigned* p, unsigned v) { return __atomic_fetch_or(p, v, __ATOMIC_RELAXED); }
static inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  const unsigned long long o = *p;
  *p += v;
  return o;
}

#include "kernels.cuh"
#include "flow_items.cuh"
#include "lower.hpp"

using namespace rteaal;

namespace {

struct Emu {
  Netlist nl, nlx;
  Lowered L;
  std::vector<uint32_t> user2x;
  DDesign d{};
  DSim s{};
  uint8_t* state = nullptr;
  std::vector<uint64_t> mem, xs;
  std::vector<uint32_t> probe_refs;
  std::vector<uint64_t> probe_prev;
  std::vector<uint8_t> act;          // activity stamps [rows][128-lane chunks]
  uint64_t act_g = 1;                // cycle number of the next step's first cycle
  bool act_force = true;             // next step's first cycle evaluates every op
  unsigned long long act_count[2] = {0, 0};
  uint32_t np = 0, err = 0;
  // FLOW form: stamped words, tables, stamps used so far
  std::vector<unsigned long long> flow_words;
  std::vector<uint32_t> flow_op, flow_ext, flow_pool;
  uint32_t flow_epoch = 0;
};

template <class T>
const T* ptr(const std::vector<T>& v) {
  static const uint64_t zero[4] = {0, 0, 0, 0};
  return v.empty() ? reinterpret_cast<const T*>(zero) : v.data();
}

// Granlund & Montgomery, PLDI 1994, Fig. 4.1 (the kernels' division by a constant)
FastDiv fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) l++;
  return FastDiv{d, (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1), l};
}

// tile_lanes = 0: the LAYER form (every phase spans all lanes); otherwise the
// TILE form's mapping (each tile of lanes runs every phase with its own lane
// base; tiles are independent, so one after another).  U: rows in flight per
// thread (the unrolled variants).
template <int V, int U>
void cycles(Emu& e, uint32_t tile_lanes, uint32_t nthreads, uint32_t ncyc) {
  const uint32_t span = tile_lanes ? tile_lanes : e.np;
  const FastDiv tpo = fastdiv(span / V);
  for (uint32_t base = 0; base < e.np; base += span)
    for (uint32_t c = 0; c < ncyc; c++) {
      if (e.s.stim_mode)
        for (uint32_t t = 0; t < nthreads; t++) stim_items<V>(e.d, e.s, make_space<V>(tpo, base, t, nthreads), c);
      for (uint32_t l = 0; l < e.d.n_layers; l++)
        for (uint32_t t = 0; t < nthreads; t++)
          eval_layer<V, U>(e.d, e.s, l, make_space<V>(tpo, base, t, nthreads), c);
      if (e.d.n_regs + e.d.n_mems)
        for (uint32_t t = 0; t < nthreads; t++) commit_items<V>(e.d, e.s, make_space<V>(tpo, base, t, nthreads), c);
      if (e.s.n_probe)
        for (uint32_t t = 0; t < nthreads; t++) probe_items<V>(e.s, make_space<V>(tpo, base, t, nthreads), c);
    }
}

// Activity-aware evaluation over all lanes (the GRID form's activity phases).
// With a multiple of 32 lane chunks per row the warps vote on hot rows
// (warp-cooperative branch: 32 host threads per warp); otherwise each thread
// checks and evaluates its own rows.
template <int V>
void cycles_act(Emu& e, uint32_t nthreads, uint32_t ncyc) {
  const FastDiv tpo = fastdiv(e.np / V);
  auto stim = [&](uint32_t c) {
    if (e.s.stim_mode)
      for (uint32_t t = 0; t < nthreads; t++) stim_items<V>(e.d, e.s, make_space<V>(tpo, 0u, t, nthreads), c);
  };
  auto edge = [&](uint32_t c) {
    if (e.d.n_regs + e.d.n_mems)
      for (uint32_t t = 0; t < nthreads; t++) commit_items<V>(e.d, e.s, make_space<V>(tpo, 0u, t, nthreads), c);
  };
  if (tpo.d % 32u != 0u) {  // each thread checks and evaluates its own rows
    for (uint32_t c = 0; c < ncyc; c++) {
      stim(c);
      for (uint32_t l = 0; l < e.d.n_layers; l++)
        for (uint32_t t = 0; t < nthreads; t++) {
          uint32_t n_eval = 0, n_skip = 0;
          threadIdx.x = t;
          eval_layer_act<V>(e.d, e.s, l, make_space<V>(tpo, 0u, t, nthreads), c, n_eval, n_skip);
          e.act_count[0] += n_eval;
          e.act_count[1] += n_skip;
        }
      edge(c);
    }
    return;
  }
  // warp-cooperative branch: 32 host threads act as the 32 lanes of a warp and
  // take the warps one after another (warps of a layer are independent); lane 0
  // runs the stimulus and clock-edge phases while the others wait
  Warp wp;
  uint32_t ev[32] = {0}, sk[32] = {0};
  std::vector<std::thread> lanes;
  for (uint32_t i = 0; i < 32; i++)
    lanes.emplace_back([&, i] {
      warp = &wp;
      for (uint32_t c = 0; c < ncyc; c++) {
        if (i == 0) stim(c);
        wp.wait();
        for (uint32_t l = 0; l < e.d.n_layers; l++) {
          for (uint32_t w0 = 0; w0 < nthreads; w0 += 32) {
            threadIdx.x = w0 + i;
            eval_layer_act<V>(e.d, e.s, l, make_space<V>(tpo, 0u, w0 + i, nthreads), c, ev[i], sk[i]);
          }
          wp.wait();
        }
        if (i == 0) edge(c);
        wp.wait();
      }
      warp = nullptr;
    });
  for (auto& th : lanes) th.join();
  for (uint32_t i = 0; i < 32; i++) {
    e.act_count[0] += ev[i];
    e.act_count[1] += sk[i];
  }
}

template <int V>
int cycles_u(Emu& e, uint32_t U, uint32_t tile_lanes, uint32_t nthreads, uint32_t ncyc) {
  switch (U) {
    case 1: cycles<V, 1>(e, tile_lanes, nthreads, ncyc); return 0;
    case 2: cycles<V, 2>(e, tile_lanes, nthreads, ncyc); return 0;
    case 4: cycles<V, 4>(e, tile_lanes, nthreads, ncyc); return 0;
    default: return -1;
  }
}

}  // namespace

// np: lanes (a power of two, every lane an instance); xs_init: [n_inputs][np].
extern "C" void* emu_create(const void* bytes, size_t nbytes, int fuse, uint32_t np, const uint64_t* xs_init) {
  Emu* e = new Emu();
  std::string err;
  if (!parse_netlist(bytes, nbytes, e->nl, err)) {
    delete e;
    return nullptr;
  }
  e->nlx = lower_clock_domains(e->nl, e->user2x);
  lower_netlist(e->nlx, e->L, fuse != 0);
  const Lowered& L = e->L;
  e->np = np;
  const size_t sbytes = (L.lane_bytes * np + 63) / 64 * 64 + 64;
  e->state = static_cast<uint8_t*>(aligned_alloc(64, sbytes));
  std::memset(e->state, 0, sbytes);
  e->mem.assign(L.mem_words_total * np + 1, 0);
  e->xs.assign(xs_init, xs_init + (size_t)L.in_width.size() * np);
  DDesign& d = e->d;
  d.meta = reinterpret_cast<const uint4*>(ptr(L.meta));
  d.dst = ptr(L.dst_ref);
  d.ext = ptr(L.ext_args);
  d.layer_off = ptr(L.layer_off);
  d.layer_ext = ptr(L.layer_ext);
  d.layer_wide = ptr(L.layer_wide);
  d.reg_src = ptr(L.reg_src);
  d.reg_ref = ptr(L.reg_ref);
  d.reg_w = ptr(L.reg_width);
  d.reg_init = ptr(L.reg_init);
  d.wport = reinterpret_cast<const uint4*>(ptr(L.wport));
  d.mem_info = reinterpret_cast<const uint4*>(ptr(L.mem_info));
  d.in_w = ptr(L.in_width);
  d.in_ref = ptr(L.in_ref);
  d.n_layers = (uint32_t)L.layer_off.size() - 1;
  d.n_regs = (uint32_t)L.reg_src.size();
  d.n_inputs = (uint32_t)L.in_width.size();
  d.n_mems = (uint32_t)(L.mem_info.size() / 4 - 1);
  d.op_base = L.op_base;
  d.reg_base = L.reg_base;
  {  // class regions of the compact layout: class 3 first, then 2, 1, 0
    const uint32_t c3 = L.class_rows[3], c2 = L.class_rows[2], c1 = L.class_rows[1];
    d.cls_off = make_uint4(8 * c3 + 4 * c2 + 2 * c1, 8 * c3 + 4 * c2, 8 * c3, 0u);
    d.cls_idx = make_uint4(c3 + c2 + c1, c3 + c2, c3, 0u);
  }
  for (size_t c = 0; c < L.const_value.size(); c++)      // constants, as at sim creation
    for (uint32_t lane = 0; lane < np; lane++) st1(e->state, L.const_ref[c], np, lane, L.const_value[c]);
  DSim& s = e->s;
  s.state = e->state;
  s.mem = e->mem.data();
  s.xs = e->xs.empty() ? nullptr : e->xs.data();
  s.n_pad = np;
  s.n_user = np;
  s.err = &e->err;
  return e;
}

// One step of the FLOW form: n_warps warps of 32 host threads (one per lane of
// a warp) run every cycle's evaluation phase concurrently and wait on one
// another's stamped words; kw items per warp and round.  The stimulus, the
// clock edge and the copies of rows no op writes run thread index by thread
// index between the phases, as the kernel's grid barriers separate them.
// Returns the error word (0: every wait ended).
extern "C" int emu_step_flow(void* p, uint32_t n_warps, uint32_t kw, uint32_t ncyc, const uint32_t* budget,
                             int reset) {
  Emu& e = *static_cast<Emu*>(p);
  e.s.budget = budget;
  e.s.uniform = ncyc;
  e.s.reset = reset;
  e.s.stim_mode = e.L.in_width.empty() ? 0 : 1;
  if (e.flow_words.empty()) {
    e.flow_words.assign((size_t)e.L.n_slots * e.np * 2 + 2, 0ull);
    flow_tables(e.L, e.flow_op, e.flow_ext, e.flow_pool);
    if (e.flow_op.empty()) e.flow_op.assign(8, 0u);
    if (e.flow_ext.empty()) e.flow_ext.push_back(0u);
    if (e.flow_pool.empty()) e.flow_pool.assign(2, 0u);
  }
  FlowArgs f{};
  f.mirror = e.flow_words.data();
  f.fop = reinterpret_cast<const uint4*>(e.flow_op.data());
  f.fext = e.flow_ext.data();
  f.fpool = reinterpret_cast<const uint2*>(e.flow_pool.data());
  f.n_in = (uint32_t)e.L.in_ref.size();
  f.n_reg = (uint32_t)e.L.reg_ref.size();
  f.n_const = (uint32_t)e.L.const_ref.size();
  f.epoch = e.flow_epoch;
  f.skew = 0;
  f.timeout_ns = 20000000000ull;
  f.off_in_smem = 0;
  f.kw = kw;
  f.span = fastdiv(e.np);
  const uint32_t T = 32 * n_warps;
  auto space = [&](uint32_t t) { return make_space<1>(f.span, 0u, t, T); };
  for (uint32_t t = 0; t < T; t++) flow_refresh(e.s, f, space(t), 0u, f.n_in + f.n_reg + f.n_const);
  for (uint32_t c = 0; c < ncyc && e.err == 0; c++) {
    for (uint32_t t = 0; t < T; t++) {
      stim_items<1>(e.d, e.s, space(t), c);
      flow_refresh(e.s, f, space(t), 0u, f.n_in);
    }
    std::vector<FlowWarp> warps(n_warps);
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < T; t++)
      th.emplace_back([&, t] {
        threadIdx.x = t;
        flow_warp = &warps[t / 32];
        flow_cycle(e.d, e.s, f, e.d.layer_off, c, t, T, f.timeout_ns);
        flow_warp = nullptr;
      });
    for (auto& x : th) x.join();
    for (uint32_t t = 0; t < T; t++) {
      commit_items<1>(e.d, e.s, space(t), c);
      flow_refresh(e.s, f, space(t), f.n_in, f.n_in + f.n_reg);
    }
  }
  e.flow_epoch += ncyc;
  return (int)e.err;
}

// One step of ncyc cycles at V lanes per item, U rows in flight, with nthreads
// thread indices per phase over all lanes (tile_lanes = 0) or per tile of
// tile_lanes lanes; budget: [np] cycles per lane (nullable: every lane runs ncyc).
extern "C" int emu_step(void* p, uint32_t V, uint32_t U, uint32_t tile_lanes, uint32_t nthreads, uint32_t ncyc,
                        const uint32_t* budget, int reset) {
  Emu& e = *static_cast<Emu*>(p);
  e.s.budget = budget;
  e.s.uniform = ncyc;
  e.s.reset = reset;
  e.s.stim_mode = e.L.in_width.empty() ? 0 : 1;   // xorshift64 stimulus
  if (tile_lanes && (e.np % tile_lanes || tile_lanes % V)) return -1;
  switch (V) {
    case 1: return cycles_u<1>(e, U, tile_lanes, nthreads, ncyc);
    case 2: return cycles_u<2>(e, U, tile_lanes, nthreads, ncyc);
    case 4: return cycles_u<4>(e, U, tile_lanes, nthreads, ncyc);
    case 8: return cycles_u<8>(e, U, tile_lanes, nthreads, ncyc);
    default: return -1;
  }
}

// Probes for the following steps (n = 0: none): mode 1 writes every cycle's
// values to out [cycles][n][np]; mode 2 appends change records {cycle | probe
// << 32, instance, value} to out (capacity records, *count = records found),
// against the probes' values as the next step begins.  -1: a signal fused away.
extern "C" int emu_probe(void* p, const uint32_t* sigs, uint32_t n, int mode, uint64_t* out, uint64_t capacity,
                         unsigned long long* count) {
  Emu& e = *static_cast<Emu*>(p);
  e.probe_refs.assign(n, 0);
  for (uint32_t i = 0; i < n; i++) {
    const uint32_t slot = e.L.sig2slot[e.user2x[sigs[i]]];
    if (slot == 0xFFFFFFFFu) return -1;
    e.probe_refs[i] = e.L.slot_ref[slot];
  }
  e.s.n_probe = n;
  e.s.probe_slot = ptr(e.probe_refs);
  e.s.probe_out = out;
  e.s.probe_changes = mode == 2;
  if (mode == 2) {
    e.probe_prev.assign((size_t)n * e.np, 0);
    for (uint32_t i = 0; i < n; i++)
      for (uint32_t lane = 0; lane < e.np; lane++)
        e.probe_prev[(size_t)i * e.np + lane] = ld1(e.state, e.probe_refs[i], e.np, lane);
    e.s.probe_prev = e.probe_prev.data();
    e.s.change_count = count;
    e.s.change_cap = capacity;
    *count = 0;
  }
  return 0;
}

// A step with activity-aware evaluation (stamps kept across steps as the
// library keeps them); stim_mode 0 holds the inputs, 1 draws xorshift64; one
// thread per lane chunk.  counts: [2] items evaluated and skipped so far.
extern "C" int emu_step_act(void* p, uint32_t V, uint32_t ncyc, const uint32_t* budget, int reset, int stim_mode,
                            unsigned long long* counts) {
  Emu& e = *static_cast<Emu*>(p);
  const uint32_t chunks = e.np / V;   // one thread per lane chunk (whole warps when 32 divide it)
  const uint32_t act_chunks = (e.np + 127) / 128;
  if (e.act.empty()) e.act.assign((size_t)e.L.n_slots * act_chunks, 0);
  e.s.budget = budget;
  e.s.uniform = ncyc;
  e.s.reset = reset;
  e.s.stim_mode = e.L.in_width.empty() ? 0 : stim_mode;   // 0: inputs held, 1: xorshift64
  e.s.act = e.act.data();
  e.s.act_chunks = act_chunks;
  e.s.act_g0 = (uint32_t)(e.act_g & 255u);
  e.s.act_force = e.act_force ? 1 : 0;
  switch (V) {
    case 1: cycles_act<1>(e, chunks, ncyc); break;
    case 2: cycles_act<2>(e, chunks, ncyc); break;
    case 4: cycles_act<4>(e, chunks, ncyc); break;
    case 8: cycles_act<8>(e, chunks, ncyc); break;
    default: return -1;
  }
  bool uneven = false;  // a lane that stopped early has an edge the next step's first cycle has not seen
  if (budget)
    for (uint32_t lane = 0; lane < e.np && !uneven; lane++) uneven = budget[lane] != ncyc;
  e.act_g += ncyc;
  e.act_force = uneven;
  e.s.act = nullptr;
  counts[0] = e.act_count[0];
  counts[1] = e.act_count[1];
  return 0;
}

// Values of a caller signal in every lane (-1: fused away).
extern "C" int emu_read(void* p, uint32_t sig, uint64_t* out) {
  Emu& e = *static_cast<Emu*>(p);
  const uint32_t slot = e.L.sig2slot[e.user2x[sig]];
  if (slot == 0xFFFFFFFFu) return -1;
  for (uint32_t lane = 0; lane < e.np; lane++) out[lane] = ld1(e.state, e.L.slot_ref[slot], e.np, lane);
  return 0;
}

extern "C" const uint64_t* emu_mem(void* p) { return static_cast<Emu*>(p)->mem.data(); }
extern "C" const uint64_t* emu_xs(void* p) { return static_cast<Emu*>(p)->xs.data(); }

extern "C" void emu_free(void* p) {
  Emu* e = static_cast<Emu*>(p);
  free(e->state);
  delete e;
}
