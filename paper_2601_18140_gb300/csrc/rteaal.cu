// rteaal.cu -- the runtime behind the C ABI (include/rteaal.h) and the kernels
// of the plain forms.
//
//   LAYER  plain form: per cycle one launch for the inputs, one per layer (the
//          kernel boundary is the LI_{i+1} <- LO_i barrier), one for the edge.
//   LAYER_GRAPH  the same launch sequence for one cycle captured as a CUDA graph
//          and replayed once per cycle (cycle index kept on the device).
//   TILE, GRID (and GRID with activity-aware evaluation) are the persistent
//          forms of persistent.cuh, STREAM the bulk-copy form of stream.cuh,
//          SPECIALIZED the run-time-compiled form of specialize.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include <chrono>

#include "kernels.cuh"
#include "host_api.hpp"
#include "lower.hpp"
#include "cluster.cuh"
#include "flow.cuh"
#include "persistent.cuh"
#include "rteaal.h"

namespace rteaal {

// ------------------------------------------------------------------ kernels

template <int V, int U>
__global__ void __launch_bounds__(256) k_layer_ops(DDesign d, DSim s, uint32_t layer, FastDiv tpo,
                                                   uint32_t cyc, const uint32_t* cyc_dev) {
  if (cyc_dev) cyc = *cyc_dev;
  const ItemSpace is = make_space<V>(tpo, 0u, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  eval_layer<V, U>(d, s, layer, is, cyc);
}

template <int V>
__global__ void __launch_bounds__(256) k_layer_stim(DDesign d, DSim s, FastDiv tpo, uint32_t cyc,
                                                    const uint32_t* cyc_dev) {
  if (cyc_dev) cyc = *cyc_dev;
  const ItemSpace is = make_space<V>(tpo, 0u, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  stim_items<V>(d, s, is, cyc);
}

template <int V>
__global__ void __launch_bounds__(256) k_layer_commit(DDesign d, DSim s, FastDiv tpo, uint32_t cyc,
                                                      const uint32_t* cyc_dev) {
  if (cyc_dev) cyc = *cyc_dev;
  const ItemSpace is = make_space<V>(tpo, 0u, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  commit_items<V>(d, s, is, cyc);
}

template <int V>
__global__ void __launch_bounds__(256) k_layer_probe(DSim s, FastDiv tpo, uint32_t cyc,
                                                     const uint32_t* cyc_dev) {
  if (cyc_dev) cyc = *cyc_dev;
  const ItemSpace is = make_space<V>(tpo, 0u, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  probe_items<V>(s, is, cyc);
}

__global__ void k_tick(uint32_t* cyc_dev) { *cyc_dev += 1u; }

}  // namespace rteaal
#include "stream.cuh"
namespace rteaal {

// compact state rows (by reference) <-> a [n][n_inst] uint64 device buffer
__global__ void k_gather_ref(const uint8_t* st, uint32_t n_pad, const uint32_t* refs, uint32_t n_rows,
                             const uint32_t* lane_of_user, uint32_t inst0, uint32_t n_inst, uint64_t* out) {
  const size_t total = (size_t)n_rows * n_inst;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)(i / n_inst), k = (uint32_t)(i % n_inst);
    const uint32_t lane = lane_of_user ? lane_of_user[inst0 + k] : inst0 + k;
    out[i] = ld1(st, refs[r], n_pad, lane);
  }
}

__global__ void k_scatter_ref(uint8_t* st, uint32_t n_pad, const uint32_t* refs, uint32_t n_rows,
                              const uint32_t* lane_of_user, uint32_t inst0, uint32_t n_inst,
                              const uint64_t* in, const uint64_t* row_mask) {
  const size_t total = (size_t)n_rows * n_inst;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)(i / n_inst), k = (uint32_t)(i % n_inst);
    const uint32_t lane = lane_of_user ? lane_of_user[inst0 + k] : inst0 + k;
    st1(st, refs[r], n_pad, lane, in[i] & row_mask[r]);
  }
}

// Fresh-sim values for the lanes of instances [inst0, inst0 + n_inst): every
// slot 0 except constant slots, memories 0, stimulus states from `xs_in`.
__global__ void k_reset_lanes(uint8_t* st, uint64_t* mem, uint64_t* xs, uint32_t n_pad,
                              const uint32_t* slot_ref, uint32_t n_slots, uint32_t const_base,
                              uint32_t n_consts, const uint64_t* const_value, uint64_t mem_words,
                              uint32_t n_inputs, const uint64_t* xs_in, const uint32_t* lane_of_user,
                              uint32_t inst0, uint32_t n_inst) {
  const size_t n_state = (size_t)n_slots * n_inst, n_mem = (size_t)mem_words * n_inst,
               n_xs = (size_t)n_inputs * n_inst;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_state + n_mem + n_xs;
       i += (size_t)gridDim.x * blockDim.x) {
    size_t j = i;
    const uint32_t k = (uint32_t)(j % n_inst);
    const uint32_t lane = lane_of_user ? lane_of_user[inst0 + k] : inst0 + k;
    if (j < n_state) {
      const uint32_t slot = (uint32_t)(j / n_inst);
      const uint64_t v = (slot >= const_base && slot < const_base + n_consts) ? const_value[slot - const_base] : 0ull;
      st1(st, slot_ref[slot], n_pad, lane, v);
    } else if ((j -= n_state) < n_mem) {
      mem[(j / n_inst) * n_pad + lane] = 0ull;
    } else {
      j -= n_mem;
      xs[(j / n_inst) * n_pad + lane] = xs_in ? xs_in[j] : 0ull;
    }
  }
}

// uint64 [row][lane] arrays (memories, stimulus states) <-> a [n][n_inst] device buffer
__global__ void k_gather(const uint64_t* src, uint32_t n_pad, const uint32_t* rows, uint32_t n_rows,
                         const uint32_t* lane_of_user, uint32_t inst0, uint32_t n_inst,
                         uint64_t* out) {
  const size_t total = (size_t)n_rows * n_inst;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)(i / n_inst), k = (uint32_t)(i % n_inst);
    const uint32_t row = rows ? rows[r] : r;
    const uint32_t lane = lane_of_user ? lane_of_user[inst0 + k] : inst0 + k;
    out[i] = src[(size_t)row * n_pad + lane];
  }
}

__global__ void k_scatter(uint64_t* dst, uint32_t n_pad, const uint32_t* rows, uint32_t n_rows,
                          const uint32_t* lane_of_user, uint32_t inst0, uint32_t n_inst,
                          const uint64_t* in, const uint64_t* row_mask) {
  const size_t total = (size_t)n_rows * n_inst;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)(i / n_inst), k = (uint32_t)(i % n_inst);
    const uint32_t row = rows ? rows[r] : r;
    const uint32_t lane = lane_of_user ? lane_of_user[inst0 + k] : inst0 + k;
    dst[(size_t)row * n_pad + lane] = in[i] & (row_mask ? row_mask[r] : ~0ull);
  }
}

// ------------------------------------------------------------------ host side

// A failed call's error stays pending in the runtime and would be returned by
// a later cudaGetLastError; it is cleared here, where it is reported.
#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cudaGetLastError();                                                                   \
      throw Error(RTEAAL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    }                                                                                       \
  } while (0)

FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{d, 0, 0};
  uint32_t l = 0;
  while ((1ull << l) < d) l++;
  f.l = l;
  f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1ull);
  return f;
}

struct Allocator {
  rteaal_allocator a{};
  bool custom = false;
  void* alloc(size_t n) {
    if (n == 0) n = 256;
    void* p = nullptr;
    if (custom) {
      p = a.alloc(n, a.ctx);
    } else if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (!p) throw Error(RTEAAL_E_NOMEM, "device allocation of " + std::to_string(n) + " bytes failed");
    return p;
  }
  void free(void* p, size_t n) {
    if (!p) return;
    if (n == 0) n = 256;
    if (custom) a.free(p, n, a.ctx);
    else cudaFree(p);
  }
};

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};

}  // namespace rteaal

using namespace rteaal;

struct rteaal_design {
  Netlist nl;                     // as loaded (the caller's signal ids)
  Netlist nlx;                    // single-clock form that is lowered and run
  std::vector<uint32_t> user2x;   // nl signal id -> nlx signal id
  Lowered L;                      // lowering of nlx
  Allocator alloc;
  int device = 0;
  int n_sms = 0;
  DDesign dd{};
  std::vector<DevBuf> bufs;
  int live_sims = 0;
  std::mutex mu;
  const uint32_t* d_slot_ref = nullptr;      // [n_slots] row reference of every slot
  const uint64_t* d_const_value = nullptr;   // [n_consts]
  uint64_t metadata_bytes = 0;

  template <typename T>
  T* upload(const std::vector<T>& v) {
    DevBuf b;
    b.n = std::max<size_t>(v.size() * sizeof(T), 16);
    b.p = alloc.alloc(b.n);
    bufs.push_back(b);
    if (!v.empty()) CK(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    metadata_bytes += b.n;
    return static_cast<T*>(b.p);
  }
  // slot of a caller's signal (0xFFFFFFFF: fused away)
  uint32_t slot_of(uint32_t sig) const { return L.sig2slot[user2x[sig]]; }

  // design-specialised kernel (compiled on first use)
  std::mutex spec_mu;
  cudaLibrary_t spec_lib = nullptr;
  cudaKernel_t spec_kernel = nullptr;
  uint64_t spec_compile_us = 0;

  ~rteaal_design() {
    if (spec_lib) cudaLibraryUnload(spec_lib);
    for (auto& b : bufs) alloc.free(b.p, b.n);
  }
};

struct rteaal_sim {
  const rteaal_design* design = nullptr;
  rteaal_design* design_mut = nullptr;
  Allocator alloc;
  uint32_t n_user = 0, n_pad = 0;
  int kernel = RTEAAL_KERNEL_AUTO;
  uint32_t tile_lanes = 0, threads = 0, ctas_per_sm = 0, unroll = 0, grid = 0;
  int V = 2;
  uint8_t* state = nullptr;          // compact rows: n_pad * lane_bytes bytes
  uint64_t* mem = nullptr;
  uint64_t* xs = nullptr;
  uint32_t* budget = nullptr;        // [n_pad]
  uint32_t* reset_lane = nullptr;    // [n_pad] per-lane leading reset cycles
  uint32_t* user_of_lane = nullptr;  // [n_pad] or null
  uint32_t* lane_of_user = nullptr;  // [n_user] or null
  uint32_t* tile_order = nullptr;    // [n_tiles]
  uint32_t* tile_cycles = nullptr;   // [n_tiles]
  uint32_t* scratch = nullptr;       // [64]: 0 err, 1 tile counter, 2-3 barrier count (u64), 4 cycle
  uint64_t* staging = nullptr;       // grown on demand (host stimulus / probe buffers)
  size_t staging_bytes = 0;
  uint32_t* probe_slots = nullptr;   // grown on demand
  uint64_t* probe_prev = nullptr;    // CHANGES probes: previous values [n][n_pad]
  size_t probe_prev_bytes = 0;
  size_t probe_slots_cap = 0;
  uint32_t* err_host = nullptr;      // pinned
  cudaEvent_t done = nullptr;
  bool pending = false;
  uint64_t device_bytes = 0;
  std::vector<uint32_t> h_lane_of_user, h_user_of_lane;
  std::vector<DevBuf> bufs;
  uint64_t barrier_timeout_ns = 2000000000ull;
  uint32_t barrier_extra = 0;        // test hook: arrivals withheld from every grid barrier
  uint32_t stream_chunk = 0;         // STREAM: lanes per item
  uint32_t stage_cap = 0;            // GRID, CLUSTER: descriptors a CTA stages in shared memory
  uint32_t cluster_ctas = 0;         // CLUSTER: CTAs per cluster
  uint32_t n_clusters = 0;           // CLUSTER: clusters resident at once
  bool resident = false;             // CLUSTER: state kept in the cluster's shared memory
  const void* cluster_fn = nullptr;  // CLUSTER: the kernel variant in use
  uint32_t res_slice = 0;            // CLUSTER resident: state bytes per CTA
  uint32_t res_smem = 0;             // CLUSTER resident: dynamic shared memory per CTA
  uint32_t last_span = 0;            // lanes the last step visited
  uint32_t last_grid = 0;            // CTAs of the last GRID / FLOW launch
  unsigned long long* flow_mirror = nullptr;  // FLOW: stamped result words, allocated on first use
  uint32_t flow_epoch = 0;           // FLOW: stamps used so far (the next cycle stamps flow_epoch + 1)
  const void* flow_fn = nullptr;     // FLOW: the kernel variant in use
  uint4* flow_op = nullptr;          // FLOW: per op {operand rows, output row}, {ctl, output ref, ext}
  uint32_t* flow_ext = nullptr;      // FLOW: operand rows of ops with more than three operands
  uint2* flow_pool = nullptr;        // FLOW: {ref, row} of inputs, registers, constants
  uint32_t flow_skew = 0;            // test hook: FLOW items wait for a stamp this far ahead
  uint32_t flow_kw = 8;              // FLOW: items a warp takes per layer and round
  // activity-aware evaluation (GRID only)
  bool activity = false;
  uint8_t* act = nullptr;            // [n_slots][act_chunks] 8-bit change stamps
  uint32_t act_chunks = 0;           // 128-lane chunks
  uint64_t act_g = 1;                // cycle number of the next step's first cycle
  bool act_force = true;             // next step's first cycle evaluates every op

  void* get(size_t n) {
    DevBuf b;
    b.n = n;
    b.p = alloc.alloc(n);
    bufs.push_back(b);
    device_bytes += n;
    return b.p;
  }
  ~rteaal_sim() {
    if (done) cudaEventDestroy(done);
    if (err_host) cudaFreeHost(err_host);
    for (auto& b : bufs) alloc.free(b.p, b.n);
  }
};

namespace {

// Lanes of a sim: a power of two up to 64 instances, else a multiple of 128
// (whole 128-lane chunks for the stream form; at most 127 idle lanes).
uint32_t pad_lanes(uint32_t n) {
  if (n <= 1) return 1;
  if (n <= 64) {
    uint32_t p = 1;
    while (p < n) p <<= 1;
    return p;
  }
  return (n + 127) / 128 * 128;
}

DSim dsim(const rteaal_sim* s) {
  DSim x{};
  x.state = s->state;
  x.mem = s->mem;
  x.xs = s->xs;
  x.n_pad = s->n_pad;
  x.n_user = s->n_user;
  x.user_of_lane = s->user_of_lane;
  x.err = s->scratch;
  if (s->activity) {
    x.act = s->act;
    x.act_chunks = s->act_chunks;
    x.act_g0 = (uint32_t)(s->act_g & 255u);
    x.act_force = s->act_force ? 1 : 0;
    x.act_count = reinterpret_cast<unsigned long long*>(s->scratch + 8);
  }
  return x;
}

// Which bounded device waits gave up (error word bits): 1 grid barrier,
// 2 stream ring barrier, 4 stream drain of its own copies after a timeout,
// 8 FLOW wait for an operand's stamp.
std::string wait_kind(uint32_t e) {
  std::string k;
  if (e & 1u) k += "grid barrier";
  if (e & 2u) k += k.empty() ? "stream ring barrier" : ", stream ring barrier";
  if (e & 4u) k += k.empty() ? "stream drain of copies in flight" : ", stream drain of copies in flight";
  if (e & 8u) k += k.empty() ? "FLOW operand stamp" : ", FLOW operand stamp";
  return k.empty() ? "unknown wait" : k;
}

void check_pending(rteaal_sim* s) {
  if (!s->pending) return;
  cudaError_t q = cudaEventQuery(s->done);
  if (q == cudaErrorNotReady) return;
  if (q != cudaSuccess) throw Error(RTEAAL_E_CUDA, std::string("previous step: ") + cudaGetErrorString(q));
  s->pending = false;
  if (const uint32_t e = *s->err_host) {
    *s->err_host = 0;
    throw Error(RTEAAL_E_TIMEOUT, std::string("a device wait timed out in a previous step (") + wait_kind(e) + ")");
  }
}

void sync_sim(rteaal_sim* s, cudaStream_t st) {
  CK(cudaStreamSynchronize(st));
  if (s->pending) {
    CK(cudaEventSynchronize(s->done));
    s->pending = false;
    if (const uint32_t e = *s->err_host) {
      *s->err_host = 0;
      throw Error(RTEAAL_E_TIMEOUT, std::string("a device wait timed out (") + wait_kind(e) + ")");
    }
  }
}

template <int V>
void launch_layer_cycle(rteaal_sim* s, const DDesign& dd, const DSim& ds, uint32_t c,
                        const uint32_t* cyc_dev, cudaStream_t st, int n_sms, uint32_t span) {
  const FastDiv tpo = make_fastdiv(span / V);
  const uint32_t threads = 256;
  auto blocks_for = [&](uint64_t items, uint32_t per_thread) {
    uint64_t b = (items + (uint64_t)threads * per_thread - 1) / ((uint64_t)threads * per_thread);
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(b, (uint64_t)n_sms * 16));
  };
  const rteaal_design* D = s->design;
  if (ds.stim_mode)
    k_layer_stim<V><<<blocks_for((uint64_t)D->L.in_width.size() * tpo.d, 1), threads, 0, st>>>(
        dd, ds, tpo, c, cyc_dev);
  const uint32_t U = s->unroll;
  for (uint32_t l = 0; l + 1 < D->L.layer_off.size(); l++) {
    const uint32_t o0 = D->L.layer_off[l], o1 = D->L.layer_off[l + 1];
    const uint64_t items = (uint64_t)(o1 - o0) * tpo.d;
    if (U >= 4)
      k_layer_ops<V, 4><<<blocks_for(items, 4), threads, 0, st>>>(dd, ds, l, tpo, c, cyc_dev);
    else if (U == 2)
      k_layer_ops<V, 2><<<blocks_for(items, 2), threads, 0, st>>>(dd, ds, l, tpo, c, cyc_dev);
    else
      k_layer_ops<V, 1><<<blocks_for(items, 1), threads, 0, st>>>(dd, ds, l, tpo, c, cyc_dev);
  }
  const uint64_t citems = (uint64_t)(D->L.reg_src.size() + (D->L.mem_info.size() / 4 - 1)) * tpo.d;
  if (citems)
    k_layer_commit<V><<<blocks_for(citems, 1), threads, 0, st>>>(dd, ds, tpo, c, cyc_dev);
  if (ds.n_probe)
    k_layer_probe<V><<<blocks_for((uint64_t)ds.n_probe * tpo.d, 1), threads, 0, st>>>(ds, tpo, c, cyc_dev);
}

// All compiled variants (tables in variants_*.cu, one translation unit each so
// that they compile in parallel).
const std::vector<Variant>& all_variants() {
  static const std::vector<Variant> all = [] {
    std::vector<Variant> v;
    for (const VariantTable& t : {variants_v8a(), variants_v8b(), variants_v8c(), variants_v8d(), variants_v4a(), variants_v4b(),
                                  variants_v4c(), variants_v2(), variants_v1()})
      v.insert(v.end(), t.v, t.v + t.n);
    return v;
  }();
  return all;
}

const std::vector<ActVariant>& all_act_variants() {
  static const std::vector<ActVariant> all = [] {
    std::vector<ActVariant> v;
    for (const ActVariantTable& t : {variants_act_a(), variants_act_b()}) v.insert(v.end(), t.v, t.v + t.n);
    return v;
  }();
  return all;
}

// Cluster variant for (V, resident): the one with exactly `threads` per CTA,
// else the first compiled for them.
const ClusterVariant* find_cluster_variant(int V, bool resident = false, uint32_t threads = 0) {
  static const ClusterVariantTable t = variants_cluster();
  for (size_t i = 0; i < t.n; i++)
    if (t.v[i].V == V && t.v[i].resident == resident && (uint32_t)t.v[i].maxt == threads) return &t.v[i];
  for (size_t i = 0; i < t.n; i++)
    if (t.v[i].V == V && t.v[i].resident == resident) return &t.v[i];
  return nullptr;
}

const ActVariant* find_act_variant(int V, uint32_t threads, uint32_t minb = 0) {
  const ActVariant* best = nullptr;
  for (const ActVariant& v : all_act_variants())
    if (v.V == V && (uint32_t)v.maxt == threads && (!minb || (uint32_t)v.minb == minb)) return &v;
  for (const ActVariant& v : all_act_variants())
    if (v.V == V && (uint32_t)v.maxt >= threads && (!best || v.maxt < best->maxt)) best = &v;
  return best;
}

// Variant for (V, U, threads): the one compiled for exactly `threads` per CTA
// (with `minb` CTAs per SM when given, else the highest occupancy target), else
// the smallest launch bound above `threads`.
const Variant* find_variant(int V, uint32_t U, uint32_t threads, uint32_t minb = 0) {
  const Variant* best = nullptr;
  for (const Variant& v : all_variants())
    if (v.V == V && (uint32_t)v.U == U && (uint32_t)v.maxt == threads && (!minb || (uint32_t)v.minb == minb) &&
        (!best || v.minb > best->minb))
      best = &v;
  if (best) return best;
  for (const Variant& v : all_variants())
    if (v.V == V && (uint32_t)v.U == U && (uint32_t)v.maxt >= threads && (!best || v.maxt < best->maxt))
      best = &v;
  return best;
}

// Lanes a launch visits: every lane up to the last one with cycles left in this
// step, rounded up to `gran` lanes (whole warps of V-lane chunks) and at most
// n_pad.  Lanes are ordered by expected cycles, so finished instances gather at
// the end and leave the span: the work per cycle follows the live instances
// (Alg. 1's iterative rank over cycles, per instance).  Lanes beyond the span
// have no cycle this step, so leaving them out changes no result.
uint32_t live_span(const rteaal_sim* s, const std::vector<uint32_t>& lane_budget, uint32_t gran) {
  uint64_t live = s->n_user;
  if (!lane_budget.empty()) {
    live = 0;
    for (size_t l = lane_budget.size(); l > 0; l--)
      if (lane_budget[l - 1]) {
        live = l;
        break;
      }
  }
  const uint64_t span = (live + gran - 1) / gran * gran;
  return (uint32_t)std::max<uint64_t>(std::min<uint64_t>(span, s->n_pad), std::min<uint64_t>(gran, s->n_pad));
}

// Persistent grid for a lane span: the configured grid, capped at what the
// widest phase over the span can occupy.
uint32_t grid_for_span(const rteaal_sim* s, uint32_t span, uint32_t V) {
  const Lowered& L = s->design->L;
  const uint64_t widest = std::max<uint64_t>(
      {(uint64_t)L.max_layer_ops, L.reg_src.size() + (L.mem_info.size() / 4 - 1), (uint64_t)L.in_width.size(), 1});
  const uint64_t items = widest * (span / V);
  return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(s->grid, (items + s->threads - 1) / s->threads));
}

// FLOW: layer offsets held in shared memory up to this many bytes (else read
// from global memory)
constexpr size_t kFlowOffSmem = 16384;

void ensure_staging(rteaal_sim* s, size_t bytes) {
  if (s->staging_bytes >= bytes) return;
  if (s->staging) {
    CK(cudaDeviceSynchronize());
    for (auto it = s->bufs.begin(); it != s->bufs.end(); ++it)
      if (it->p == s->staging) {
        s->alloc.free(it->p, it->n);
        s->device_bytes -= it->n;
        s->bufs.erase(it);
        break;
      }
  }
  s->staging = static_cast<uint64_t*>(s->get(bytes));
  s->staging_bytes = bytes;
}

void ensure_probe_slots(rteaal_sim* s, size_t n) {
  if (s->probe_slots_cap >= n) return;
  s->probe_slots = static_cast<uint32_t*>(s->get(std::max<size_t>(n, 64) * 4));
  s->probe_slots_cap = std::max<size_t>(n, 64);
}

}  // namespace

// ================================================================== C ABI

RT_EXPORT int rteaal_design_load(const void* netlist, size_t nbytes, const rteaal_load_opts* opts,
                                 rteaal_design** out) {
  return guarded([&] {
    require(netlist && out, "rteaal_design_load: null argument");
    *out = nullptr;
    auto* d = new rteaal_design();
    try {
      std::string err;
      if (!parse_netlist(netlist, nbytes, d->nl, err)) throw Error(RTEAAL_E_FORMAT, err);
      if (opts && opts->allocator) {
        d->alloc.a = *opts->allocator;
        d->alloc.custom = d->alloc.a.alloc && d->alloc.a.free;
      }
      if (opts && opts->device >= 0) CK(cudaSetDevice(opts->device));
      CK(cudaGetDevice(&d->device));
      CK(cudaDeviceGetAttribute(&d->n_sms, cudaDevAttrMultiProcessorCount, d->device));
      d->nlx = lower_clock_domains(d->nl, d->user2x);
      lower_netlist(d->nlx, d->L, opts && opts->fuse_mux_chains);
      const Lowered& L = d->L;
      DDesign& dd = d->dd;
      static_assert(sizeof(OpMeta) == sizeof(uint4), "descriptor is 16 bytes");
      dd.meta = reinterpret_cast<const uint4*>(d->upload(L.meta));
      dd.dst = d->upload(L.dst_ref);
      dd.reg_ref = d->upload(L.reg_ref);
      dd.in_ref = d->upload(L.in_ref);
      dd.ext = d->upload(L.ext_args);
      dd.layer_off = d->upload(L.layer_off);
      dd.layer_ext = d->upload(L.layer_ext);
      dd.layer_wide = d->upload(L.layer_wide);
      dd.reg_src = d->upload(L.reg_src);
      dd.reg_w = d->upload(L.reg_width);
      dd.reg_init = d->upload(L.reg_init);
      dd.wport = reinterpret_cast<const uint4*>(d->upload(L.wport));
      dd.mem_info = reinterpret_cast<const uint4*>(d->upload(L.mem_info));
      dd.in_w = d->upload(L.in_width);
      d->d_slot_ref = d->upload(L.slot_ref);
      d->d_const_value = d->upload(L.const_value);
      dd.n_layers = (uint32_t)L.layer_off.size() - 1;
      dd.n_regs = (uint32_t)L.reg_src.size();
      dd.n_inputs = (uint32_t)L.in_width.size();
      dd.n_mems = (uint32_t)(L.mem_info.size() / 4 - 1);
      dd.op_base = L.op_base;
      dd.reg_base = L.reg_base;
      {  // class regions of the compact layout: class 3 first, then 2, 1, 0
        const uint64_t c3 = L.class_rows[3], c2 = L.class_rows[2], c1 = L.class_rows[1];
        dd.cls_off = make_uint4((uint32_t)(8 * c3 + 4 * c2 + 2 * c1), (uint32_t)(8 * c3 + 4 * c2),
                                (uint32_t)(8 * c3), 0u);
        dd.cls_idx = make_uint4((uint32_t)(c3 + c2 + c1), (uint32_t)(c3 + c2), (uint32_t)c3, 0u);
      }
    } catch (...) {
      delete d;
      throw;
    }
    *out = d;
  });
}

RT_EXPORT int rteaal_design_info(const rteaal_design* d, rteaal_design_stats* o) {
  return guarded([&] {
    require(d && o, "rteaal_design_info: null argument");
    fill_stats(d->nl, d->L, d->metadata_bytes, o);
  });
}

RT_EXPORT int rteaal_design_signals(const rteaal_design* d, uint8_t* present, uint64_t n) {
  return guarded([&] {
    require(d && present, "rteaal_design_signals: null argument");
    require(n == d->nl.n_signals(), "rteaal_design_signals: n_signals differs from the design's");
    for (uint64_t i = 0; i < n; i++) present[i] = d->slot_of((uint32_t)i) != 0xFFFFFFFFu;
  });
}

RT_EXPORT int rteaal_design_free(rteaal_design* d) {
  if (!d) return RTEAAL_OK;
  {
    std::lock_guard<std::mutex> g(d->mu);
    if (d->live_sims > 0) {
      last_error() = "rteaal_design_free: simulations created from this design are still alive";
      return RTEAAL_E_BUSY;
    }
  }
  delete d;
  return RTEAAL_OK;
}

RT_EXPORT uint64_t rteaal_sim_footprint(const rteaal_design* d, uint32_t n) {
  if (!d || n == 0) return 0;
  const uint64_t np = pad_lanes(n);
  const Lowered& L = d->L;
  return np * (L.lane_bytes + 8ull * (L.mem_words_total + L.in_width.size())) + np * 4ull * 5 +
         (uint64_t)n * 4 + 4096;
}

namespace {


constexpr uint32_t kSpecMaxOps = 16384;
constexpr uint32_t kSpecThreads = 128;
constexpr uint32_t kSpecOptimizeOps = 4096;  // NVVM optimiser on up to this many ops

// Generate and compile (NVRTC, sm_103a) the design-specialised kernel of a
// lowered netlist; host only.
std::vector<char> build_specialized(const Netlist& nlx, const Lowered& L) {
  if (nlx.no > kSpecMaxOps)
    throw Error(RTEAAL_E_UNSUPPORTED, "design-specialised kernel: more than 16,384 ops (compile time grows superlinearly)");
  const std::string src = specialized_source(nlx, L);
  std::vector<char> cubin;
  std::string log;
  if (!compile_specialized(src, "sm_103a", nlx.no <= kSpecOptimizeOps, cubin, log))
    throw Error(RTEAAL_E_CUDA, "design-specialised kernel: compile failed: " + log.substr(0, 2000));
  return cubin;
}

// Generate, compile and load the design-specialised kernel once per design.
void ensure_specialized(rteaal_design* d) {
  std::lock_guard<std::mutex> g(d->spec_mu);
  if (d->spec_kernel) return;
  const auto t0 = std::chrono::steady_clock::now();
  const std::vector<char> cubin = build_specialized(d->nlx, d->L);
  CK(cudaSetDevice(d->device));
  CK(cudaLibraryLoadData(&d->spec_lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
  CK(cudaLibraryGetKernel(&d->spec_kernel, d->spec_lib, "rteaal_spec"));
  d->spec_compile_us = (uint64_t)std::chrono::duration_cast<std::chrono::microseconds>(
                           std::chrono::steady_clock::now() - t0).count();
}

// Shared-memory descriptor staging of the GRID form (persistent.cuh): a CTA
// stages, per layer, the descriptors of the rows its threads evaluate --
// at most ceil(layer rows / per) steps of span rows, per = threads / lane
// chunks and span <= ceil(CTA threads / lane chunks) + 1.  Capped so that the
// CTAs of an SM share at most ~200 KB; layers beyond the cap read their
// descriptors from global memory.
constexpr uint32_t kStageBytes = 20;       // 16-byte descriptor + 4-byte output row
constexpr uint32_t kStageMax = 2304;       // at most 46 KB per CTA (no opt-in needed)
uint32_t stage_capacity(uint32_t chunks, uint32_t grid, uint32_t threads, uint32_t max_layer_ops,
                        uint32_t ctas_per_sm) {
  const uint64_t nthreads = (uint64_t)grid * threads;
  if (chunks == 0 || nthreads < chunks || max_layer_ops == 0) return 0;
  const uint64_t per = nthreads / chunks;
  const uint64_t span = (threads + chunks - 1) / chunks + 1;
  const uint64_t rows = (max_layer_ops + per - 1) / per * span;
  const uint64_t budget = 200ull * 1024 / std::max<uint32_t>(ctas_per_sm, 1) / kStageBytes;
  return (uint32_t)std::min<uint64_t>({rows, kStageMax, budget});
}

// Validate and apply a launch configuration (never changes results).
// Dynamic shared memory of the cluster kernels besides the resident state: two
// staging buffers of descriptors and output rows, and the layer table.
uint64_t cluster_table_smem(uint32_t stage, uint32_t n_layers) {
  return 2ull * stage * kStageBytes + 4ull * (3ull * n_layers + 1);
}

// Let a kernel take up to the opt-in shared memory less its static part.
int allow_max_smem(const void* fn, int device) {
  int optin = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  cudaFuncAttributes fa{};
  CK(cudaFuncGetAttributes(&fa, fn));
  const int dyn_max = std::max(optin - (int)fa.sharedSizeBytes, 0);
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
  return dyn_max;
}

// Resident cluster form (cluster.cuh): the smallest slice layout that fits,
// for the given cluster size (0: the first of 8, 16, 4, 2 that fits).  Returns
// the cluster size, 0 if none fits; sets the slice, staging capacity and
// shared memory per CTA.
uint32_t plan_resident(rteaal_sim* s, const ClusterVariant* cv, uint32_t cluster_ctas, uint32_t& slice,
                       uint32_t& stage, uint32_t& smem) {
  const Lowered& L = s->design->L;
  const uint64_t bytes = (uint64_t)s->n_pad * L.lane_bytes;
  constexpr uint64_t kBudget = 220 * 1024;
  if (!cv) return 0;
  const void* fn = cv->fn;
  const uint32_t nthr = (uint32_t)cv->maxt;
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  for (uint32_t cs : {8u, 16u, 4u, 2u}) {
    if (cluster_ctas && cs != cluster_ctas) continue;
    const uint64_t S = ((bytes + cs - 1) / cs + 15) / 16 * 16;
    if (S + 16 > kBudget) continue;
    const uint64_t table = cluster_table_smem(0, (uint32_t)(L.layer_off.size() - 1));
    if (S + table > kBudget) continue;
    uint64_t st = stage_capacity(s->n_pad, cs, nthr, L.max_layer_ops, 1);
    st = std::min<uint64_t>(st, (kBudget - S - table) / (2 * kStageBytes));
    const uint64_t sm = S + cluster_table_smem((uint32_t)st, (uint32_t)(L.layer_off.size() - 1));
    // a sim's launch asks for its own size, at most the opt-in maximum
    if (sm > (uint64_t)allow_max_smem(fn, s->design->device)) continue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(nthr);
    cfg.dynamicSmemBytes = sm;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      ncl = 0;
    }
    if (ncl < 1) continue;
    slice = (uint32_t)S;
    stage = (uint32_t)st;
    smem = (uint32_t)sm;
    return cs;
  }
  return 0;
}

void configure(rteaal_sim* s, int kernel, uint32_t tile_lanes, uint32_t threads, uint32_t ctas_per_sm,
               uint32_t unroll, uint32_t lanes_per_thread, uint32_t cluster_ctas = 0, int cluster_resident = 0) {
  const uint32_t tile_lanes_in = tile_lanes;  // as asked (FLOW: items per warp)
  if (kernel == RTEAAL_KERNEL_AUTO)
    kernel = s->activity ? RTEAAL_KERNEL_GRID : s->n_pad >= 64 ? RTEAAL_KERNEL_TILE : RTEAAL_KERNEL_LAYER;
  if (s->activity && kernel != RTEAAL_KERNEL_GRID)
    throw Error(RTEAAL_E_UNSUPPORTED, "activity-aware evaluation runs with the GRID kernel only");
  if (s->activity && unroll > 1)
    throw Error(RTEAAL_E_UNSUPPORTED, "activity-aware evaluation has no unrolled variants");
  require(kernel >= RTEAAL_KERNEL_LAYER && kernel <= RTEAAL_KERNEL_FLOW, "unknown kernel");
  if (kernel == RTEAAL_KERNEL_CLUSTER && !tile_lanes)  // a cluster tile: all lanes of a small sim, else 256 / 128
    tile_lanes = s->n_pad <= 256 ? s->n_pad : s->n_pad % 256 == 0 ? 256u : 128u;
  if (!unroll) unroll = 1;
  require(unroll == 1 || unroll == 2 || unroll == 4, "unroll must be 1, 2 or 4");
  if (!threads) threads = 512;
  require(threads % 32 == 0 && threads >= 32 && threads <= 1024, "threads must be a multiple of 32 in [32, 1024]");
  if (!tile_lanes) tile_lanes = std::min<uint32_t>(16, s->n_pad);
  require(lanes_per_thread == 0 || lanes_per_thread == 1 || lanes_per_thread == 2 || lanes_per_thread == 4 ||
              lanes_per_thread == 8,
          "lanes_per_thread must be 1, 2, 4 or 8");
  uint32_t span = s->n_pad;  // lanes that one V-lane chunk must divide
  if (kernel == RTEAAL_KERNEL_CLUSTER) {
    require(tile_lanes >= 1 && s->n_pad % tile_lanes == 0, "cluster tile_lanes must divide the padded lane count");
    span = tile_lanes;
  }
  if (kernel == RTEAAL_KERNEL_TILE) {
    require(tile_lanes >= 1 && tile_lanes <= 64 && (tile_lanes & (tile_lanes - 1)) == 0,
            "tile_lanes must be a power of two <= 64");
    require(s->n_pad % tile_lanes == 0, "tile_lanes must divide the padded lane count");
    span = tile_lanes;
  }
  int V = (int)lanes_per_thread;
  if (!V) {  // widest V that divides the span and (persistent forms) has a compiled variant
    const bool persistent = kernel == RTEAAL_KERNEL_TILE || kernel == RTEAAL_KERNEL_GRID;
    if (kernel == RTEAAL_KERNEL_CLUSTER) {
      for (int c : {8, 4, 2, 1})
        if (span % (uint32_t)c == 0 && find_cluster_variant(c, false)) {
          V = c;
          break;
        }
    } else {
      for (int c : {4, 2, 1, 8})
        if (span % (uint32_t)c == 0 && (!persistent || find_variant(c, unroll ? unroll : 1, threads ? threads : 512))) {
          V = c;
          break;
        }
    }
    if (!V) V = 1;
  }
  require(span % (uint32_t)V == 0, "lanes_per_thread must divide the lanes of a tile / the padded lane count");
  uint32_t grid = 0, stage = 0;
  if (kernel == RTEAAL_KERNEL_LAYER || kernel == RTEAAL_KERNEL_LAYER_GRAPH) threads = 256;
  if (kernel == RTEAAL_KERNEL_SPECIALIZED) {
    ensure_specialized(s->design_mut);
    threads = kSpecThreads;
    V = 1;
    unroll = 1;
    ctas_per_sm = 0;
    grid = (uint32_t)((s->n_pad + kSpecThreads - 1) / kSpecThreads);
  } else if (kernel == RTEAAL_KERNEL_CLUSTER && cluster_resident >= 0 && tile_lanes == s->n_pad && s->n_pad <= 64 &&
             (plan_resident(s, find_cluster_variant(1, true, threads), cluster_ctas, s->res_slice, stage,
                            s->res_smem) != 0 ||
              cluster_resident > 0)) {
    // the whole state in the cluster's distributed shared memory, one lane per thread
    const ClusterVariant* cv = find_cluster_variant(1, true, threads);
    const uint32_t cs = plan_resident(s, cv, cluster_ctas, s->res_slice, stage, s->res_smem);
    if (!cs) throw Error(RTEAAL_E_UNSUPPORTED, "cluster form: the state does not fit the cluster's shared memory");
    s->resident = true;
    s->cluster_fn = cv->fn;
    s->cluster_ctas = cs;
    s->n_clusters = 1;
    V = 1;
    threads = (uint32_t)cv->maxt;
    unroll = 1;
    ctas_per_sm = 1;
    grid = cs;
  } else if (kernel == RTEAAL_KERNEL_CLUSTER) {
    s->resident = false;
    const ClusterVariant* cv = find_cluster_variant(V, false, threads);
    if (!cv) throw Error(RTEAAL_E_UNSUPPORTED, "no compiled cluster variant for V=" + std::to_string(V));
    s->cluster_fn = cv->fn;
    threads = (uint32_t)cv->maxt;
    unroll = 1;
    require(cluster_ctas == 0 || (cluster_ctas >= 1 && cluster_ctas <= 16), "cluster_ctas must be in 1..16");
    CK(cudaFuncSetAttribute(cv->fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    const Lowered& L = s->design->L;
    const uint32_t n_layers = (uint32_t)(L.layer_off.size() - 1);
    const int dyn_max = allow_max_smem(cv->fn, s->design->device);
    uint32_t best_cs = 0, best_ncl = 0;
    for (uint32_t cs : {16u, 8u, 4u, 2u, 1u}) {
      if (cluster_ctas && cs != cluster_ctas) continue;
      stage = stage_capacity(tile_lanes / (uint32_t)V, cs, threads, L.max_layer_ops, 1);
      while (stage && cluster_table_smem(stage, n_layers) > (uint64_t)dyn_max) stage /= 2;
      if (cluster_table_smem(stage, n_layers) > (uint64_t)dyn_max) continue;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cs;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(threads);
      cfg.dynamicSmemBytes = cluster_table_smem(stage, n_layers);
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, cv->fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        ncl = 0;
      }
      if (ncl > 0) {
        best_cs = cs;
        best_ncl = (uint32_t)ncl;
        break;
      }
    }
    if (!best_cs) throw Error(RTEAAL_E_UNSUPPORTED, "cluster kernel cannot be resident");
    stage = stage_capacity(tile_lanes / (uint32_t)V, best_cs, threads, L.max_layer_ops, 1);
    while (stage && cluster_table_smem(stage, n_layers) > (uint64_t)dyn_max) stage /= 2;
    s->cluster_ctas = best_cs;
    s->n_clusters = std::min<uint32_t>(best_ncl, s->n_pad / tile_lanes);
    ctas_per_sm = 1;
    grid = s->n_clusters * best_cs;
  } else if (kernel == RTEAAL_KERNEL_FLOW) {
    // one lane per item; a grid sized to the widest phase (threads beyond it
    // only add arrivals to the barriers around the stimulus and the edge)
    const FlowVariantTable ft = variants_flow();
    const FlowVariant* fv = nullptr;
    for (size_t i = 0; i < ft.n; i++)
      if ((uint32_t)ft.v[i].maxt == threads) fv = &ft.v[i];
    if (!fv)
      for (size_t i = 0; i < ft.n; i++)
        if (ft.v[i].maxt == 128) fv = &ft.v[i];
    require(fv != nullptr, "no compiled FLOW variant");
    s->flow_fn = fv->fn;
    // tile_lanes: items a warp takes per layer (1..32; 0 = 8)
    require(tile_lanes_in <= 32, "FLOW: tile_lanes (items per warp) must be in 1..32");
    s->flow_kw = tile_lanes_in ? tile_lanes_in : 8u;
    tile_lanes = s->flow_kw;
    threads = (uint32_t)fv->maxt;
    V = 1;
    unroll = 1;
    int occ = 0;  // with the most shared memory a launch asks for (the layer offsets)
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fv->fn, (int)threads, kFlowOffSmem));
    require(occ >= 1, "FLOW kernel cannot be resident");
    ctas_per_sm = (uint32_t)occ;
    const Lowered& L = s->design->L;
    const uint64_t widest = std::max<uint64_t>(
        {(uint64_t)L.max_layer_ops, L.reg_src.size() + (L.mem_info.size() / 4 - 1), (uint64_t)L.in_width.size(), 1});
    grid = (uint32_t)std::min<uint64_t>((uint64_t)occ * s->design->n_sms,
                                        (std::max<uint64_t>(widest, (uint64_t)L.max_layer_ops * 32 / s->flow_kw) *
                                             s->n_pad + threads - 1) / threads);
  } else if (kernel == RTEAAL_KERNEL_STREAM) {
    // one CTA of STREAM_WARPS warps per SM; items of 256 lanes (128 when the
    // lane count is an odd multiple of 128); every warp keeps one chunk
    if (s->n_pad % 128 != 0)
      throw Error(RTEAAL_E_UNSUPPORTED, "stream kernel needs a multiple of 128 lanes");
    const uint32_t half = s->n_pad % 256 == 0 ? 2u : 1u;
    s->stream_chunk = 128u * half;
    if ((uint64_t)s->design->n_sms * STREAM_WARPS < s->n_pad / s->stream_chunk)
      throw Error(RTEAAL_E_UNSUPPORTED, "stream kernel: more lane chunks than warps");
    V = (int)STREAM_V;
    threads = 32 * STREAM_WARPS;
    unroll = 1;
    const void* fn = half == 2 ? (const void*)k_stream<2> : (const void*)k_stream<1>;
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stream_smem_bytes()));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, (int)threads, stream_smem_bytes()));
    require(occ >= 1, "stream kernel cannot be resident");
    ctas_per_sm = 1;
    grid = (uint32_t)s->design->n_sms;
  } else if (kernel == RTEAAL_KERNEL_GRID && s->activity) {
    if (!lanes_per_thread && !find_act_variant(V, threads)) V = 4;
    const ActVariant* v = find_act_variant(V, threads, ctas_per_sm);
    if (!v)  // no variant for these threads: the first one compiled for this V, at its block size
      for (const ActVariant& c : all_act_variants())
        if (c.V == V) {
          v = &c;
          threads = (uint32_t)c.maxt;
          break;
        }
    if (!v) throw Error(RTEAAL_E_UNSUPPORTED, "no compiled activity-aware variant for V=" + std::to_string(V) +
                                                  " threads=" + std::to_string(threads));
    require(span % (uint32_t)V == 0, "lanes_per_thread must divide the padded lane count");
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v->grid, (int)threads, 0));
    require(occ >= 1, "kernel cannot be resident with these threads");
    ctas_per_sm = ctas_per_sm ? std::min<uint32_t>(ctas_per_sm, (uint32_t)occ) : (uint32_t)occ;
    grid = ctas_per_sm * (uint32_t)s->design->n_sms;
    if ((uint64_t)grid * threads < s->n_pad / (uint32_t)V)
      throw Error(RTEAAL_E_UNSUPPORTED, "activity-aware evaluation needs a thread per lane chunk");
  } else if (kernel == RTEAAL_KERNEL_TILE || kernel == RTEAAL_KERNEL_GRID) {
    const Variant* v = find_variant(V, unroll, threads, ctas_per_sm);
    if (!v) throw Error(RTEAAL_E_UNSUPPORTED, "no compiled kernel variant for V=" + std::to_string(V) +
                                                  " unroll=" + std::to_string(unroll) +
                                                  " threads=" + std::to_string(threads));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel == RTEAAL_KERNEL_GRID ? v->grid : v->tile,
                                                     (int)threads, 0));
    require(occ >= 1, "kernel cannot be resident with these threads");
    ctas_per_sm = ctas_per_sm ? std::min<uint32_t>(ctas_per_sm, (uint32_t)occ) : (uint32_t)occ;
    grid = ctas_per_sm * (uint32_t)s->design->n_sms;
    if (kernel == RTEAAL_KERNEL_TILE) grid = std::min<uint32_t>(grid, s->n_pad / tile_lanes);
    if (kernel == RTEAAL_KERNEL_GRID) {
      // CTAs beyond what the widest phase (a layer, or the register commit) can
      // occupy only add arrivals to every grid barrier: few lanes (one instance)
      // then run on a grid sized to the work
      const Lowered& L = s->design->L;
      const uint64_t widest = std::max<uint64_t>(L.max_layer_ops, L.reg_src.size() + (L.mem_info.size() / 4 - 1));
      const uint64_t items = std::max<uint64_t>(widest, 1) * (s->n_pad / V);
      grid = (uint32_t)std::min<uint64_t>(grid, (items + threads - 1) / threads);
      stage = stage_capacity(s->n_pad / (uint32_t)V, grid, threads, L.max_layer_ops, ctas_per_sm);
      if (stage) {  // the staged descriptors must not lower the residency the grid counts on
        int occ2 = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, v->grid, (int)threads, stage * kStageBytes));
        if ((uint32_t)occ2 < ctas_per_sm) stage = 0;
      }
    }
  } else {
    ctas_per_sm = 0;
  }
  s->kernel = kernel;
  s->stage_cap = stage;
  s->tile_lanes = tile_lanes;
  s->threads = threads;
  s->ctas_per_sm = ctas_per_sm;
  s->unroll = unroll;
  s->V = V;
  s->grid = grid;
}

uint32_t opt_lanes(const rteaal_sim_opts* o) { return o ? o->lanes_per_thread : 0; }

}  // namespace

RT_EXPORT int rteaal_design_specialize(rteaal_design* d, uint64_t* compile_us) {
  return guarded([&] {
    require(d, "rteaal_design_specialize: null design");
    ensure_specialized(d);
    if (compile_us) *compile_us = d->spec_compile_us;
  });
}

RT_EXPORT int rteaal_design_specialized_source(const void* netlist, size_t nbytes, const rteaal_load_opts* opts,
                                               char* out, size_t capacity, size_t* out_bytes) {
  return guarded([&] {
    require(netlist && out_bytes, "rteaal_design_specialized_source: null argument");
    Netlist nl;
    std::string err;
    if (!parse_netlist(netlist, nbytes, nl, err)) throw Error(RTEAAL_E_FORMAT, err);
    std::vector<uint32_t> user2x;
    const Netlist nlx = lower_clock_domains(nl, user2x);
    Lowered L;
    lower_netlist(nlx, L, opts && opts->fuse_mux_chains);
    const std::string src = specialized_source(nlx, L);
    *out_bytes = src.size();
    if (out) {
      require(capacity >= src.size(), "rteaal_design_specialized_source: output buffer too small");
      std::memcpy(out, src.data(), src.size());
    }
  });
}

RT_EXPORT int rteaal_design_specialize_host(const void* netlist, size_t nbytes, const rteaal_load_opts* opts,
                                            uint64_t* cubin_bytes, uint64_t* compile_us) {
  return guarded([&] {
    require(netlist, "rteaal_design_specialize_host: null netlist");
    Netlist nl;
    std::string err;
    if (!parse_netlist(netlist, nbytes, nl, err)) throw Error(RTEAAL_E_FORMAT, err);
    std::vector<uint32_t> user2x;
    const Netlist nlx = lower_clock_domains(nl, user2x);
    Lowered L;
    lower_netlist(nlx, L, opts && opts->fuse_mux_chains);
    const auto t0 = std::chrono::steady_clock::now();
    const std::vector<char> cubin = build_specialized(nlx, L);
    if (cubin_bytes) *cubin_bytes = cubin.size();
    if (compile_us)
      *compile_us = (uint64_t)std::chrono::duration_cast<std::chrono::microseconds>(
                        std::chrono::steady_clock::now() - t0).count();
  });
}

RT_EXPORT int rteaal_sim_create(const rteaal_design* d, uint32_t n_instances, const rteaal_sim_opts* opts,
                                rteaal_sim** out) {
  return guarded([&] {
    require(d && out && n_instances >= 1, "rteaal_sim_create: bad argument");
    *out = nullptr;
    auto* s = new rteaal_sim();
    try {
      s->design = d;
      s->design_mut = const_cast<rteaal_design*>(d);
      if (opts && opts->allocator) {
        s->alloc.a = *opts->allocator;
        s->alloc.custom = s->alloc.a.alloc && s->alloc.a.free;
      }
      CK(cudaSetDevice(d->device));
      s->n_user = n_instances;
      s->n_pad = pad_lanes(n_instances);
      s->activity = opts && opts->activity;
      configure(s, opts ? opts->kernel : 0, opts ? opts->tile_lanes : 0, opts ? opts->threads : 0,
                opts ? opts->ctas_per_sm : 0, opts ? opts->unroll : 0, opt_lanes(opts), opts ? opts->cluster_ctas : 0,
                opts ? opts->cluster_resident : 0);
      if (const char* e = getenv("RTEAAL_TEST_WITHHOLD_ARRIVAL")) s->barrier_extra = (uint32_t)atoi(e);
      if (const char* e = getenv("RTEAAL_TEST_FLOW_STAMP_SKEW")) s->flow_skew = (uint32_t)atoi(e);
      if (const char* e = getenv("RTEAAL_BARRIER_TIMEOUT_NS")) s->barrier_timeout_ns = strtoull(e, nullptr, 10);

      const Lowered& L = d->L;
      const size_t np = s->n_pad;
      s->state = static_cast<uint8_t*>(s->get(std::max<size_t>(np * L.lane_bytes, 16)));
      s->mem = static_cast<uint64_t*>(s->get(std::max<size_t>(np * 8 * L.mem_words_total, 16)));
      s->xs = static_cast<uint64_t*>(s->get(std::max<size_t>(np * 8 * L.in_width.size(), 16)));
      s->budget = static_cast<uint32_t*>(s->get(np * 4));
      s->reset_lane = static_cast<uint32_t*>(s->get(np * 4));
      s->tile_order = static_cast<uint32_t*>(s->get(np * 4));   // room for any tile size
      s->tile_cycles = static_cast<uint32_t*>(s->get(np * 4));
      s->scratch = static_cast<uint32_t*>(s->get(256));
      CK(cudaMemset(s->state, 0, std::max<size_t>(np * L.lane_bytes, 16)));
      CK(cudaMemset(s->mem, 0, std::max<size_t>(np * 8 * L.mem_words_total, 16)));
      CK(cudaMemset(s->xs, 0, std::max<size_t>(np * 8 * L.in_width.size(), 16)));
      CK(cudaMemset(s->scratch, 0, 256));
      if (s->activity) {
        s->act_chunks = (uint32_t)((np + 127) / 128);
        const size_t ab = std::max<size_t>((size_t)L.n_slots * s->act_chunks, 16);
        s->act = static_cast<uint8_t*>(s->get(ab));
        CK(cudaMemset(s->act, 0, ab));
      }
      // lane order: descending expected cycles (stable), so tiles retire together
      s->h_user_of_lane.assign(np, 0xFFFFFFFFu);
      s->h_lane_of_user.resize(n_instances);
      std::vector<uint32_t> ord(n_instances);
      std::iota(ord.begin(), ord.end(), 0u);
      if (opts && opts->expected_cycles) {
        const uint32_t* ec = opts->expected_cycles;
        std::stable_sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) { return ec[a] > ec[b]; });
      }
      bool identity = true;
      for (uint32_t l = 0; l < n_instances; l++) {
        s->h_user_of_lane[l] = ord[l];
        s->h_lane_of_user[ord[l]] = l;
        identity &= ord[l] == l;
      }
      if (!identity) {
        s->user_of_lane = static_cast<uint32_t*>(s->get(np * 4));
        s->lane_of_user = static_cast<uint32_t*>(s->get((size_t)n_instances * 4));
        CK(cudaMemcpy(s->user_of_lane, s->h_user_of_lane.data(), np * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(s->lane_of_user, s->h_lane_of_user.data(), (size_t)n_instances * 4, cudaMemcpyHostToDevice));
      }
      // constants: every lane (padded ones too) holds the value
      if (!L.const_value.empty()) {
        const size_t nc = L.const_value.size();
        std::vector<uint64_t> h(nc * np), ones(nc, ~0ull);
        for (size_t c = 0; c < nc; c++)
          for (size_t l = 0; l < np; l++) h[c * np + l] = L.const_value[c];
        const size_t bytes = h.size() * 8 + nc * 12 + 64;
        char* tmp = static_cast<char*>(s->alloc.alloc(bytes));
        uint64_t* dv = reinterpret_cast<uint64_t*>(tmp);
        uint64_t* dm = dv + h.size();
        uint32_t* dr = reinterpret_cast<uint32_t*>(dm + nc);
        cudaError_t e = cudaMemcpy(dv, h.data(), h.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dm, ones.data(), nc * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dr, L.const_ref.data(), nc * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
          k_scatter_ref<<<(unsigned)std::min<size_t>((h.size() + 255) / 256, 4096), 256>>>(
              s->state, s->n_pad, dr, (uint32_t)nc, nullptr, 0, s->n_pad, dv, dm);
          e = cudaDeviceSynchronize();
        }
        s->alloc.free(tmp, bytes);
        CK(e);
      }
      if (opts && opts->xorshift_seed && !L.in_width.empty()) {
        std::vector<uint64_t> h(L.in_width.size() * np, 0);
        for (size_t j = 0; j < L.in_width.size(); j++)
          for (uint32_t u = 0; u < n_instances; u++)
            h[j * np + s->h_lane_of_user[u]] = opts->xorshift_seed[j * n_instances + u];
        CK(cudaMemcpy(s->xs, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
      }
      CK(cudaMallocHost(&s->err_host, 64));
      *s->err_host = 0;
      CK(cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming));
      {
        std::lock_guard<std::mutex> g(s->design_mut->mu);
        s->design_mut->live_sims++;
      }
    } catch (...) {
      delete s;
      throw;
    }
    *out = s;
  });
}

RT_EXPORT int rteaal_sim_configure(rteaal_sim* s, const rteaal_sim_opts* o) {
  return guarded([&] {
    require(s && o, "rteaal_sim_configure: null argument");
    CK(cudaSetDevice(s->design->device));
    configure(s, o->kernel, o->tile_lanes, o->threads, o->ctas_per_sm, o->unroll, o->lanes_per_thread,
              o->cluster_ctas, o->cluster_resident);
  });
}

RT_EXPORT int rteaal_sim_info(const rteaal_sim* s, rteaal_sim_stats* o) {
  return guarded([&] {
    require(s && o, "rteaal_sim_info: null argument");
    o->n_instances = s->n_user;
    o->n_lanes = s->n_pad;
    o->device_bytes = s->device_bytes;
    o->kernel = s->kernel;
    o->tile_lanes = s->tile_lanes;
    o->threads = s->threads;
    o->ctas_per_sm = s->ctas_per_sm;
    o->unroll = s->unroll;
    o->grid = s->grid;
    o->lanes_per_thread = (uint32_t)s->V;
    o->activity = s->activity ? 1 : 0;
    o->last_span = s->last_span;
    o->last_grid = s->last_grid;
    o->cluster_ctas = s->kernel == RTEAAL_KERNEL_CLUSTER ? s->cluster_ctas : 0;
    o->cluster_resident = s->kernel == RTEAAL_KERNEL_CLUSTER && s->resident ? 1 : 0;
  });
}

RT_EXPORT int rteaal_sim_activity(rteaal_sim* s, uint64_t* evaluated, uint64_t* skipped, void* stream) {
  return guarded([&] {
    require(s && evaluated && skipped, "rteaal_sim_activity: null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(s->design->device));
    sync_sim(s, st);
    uint64_t c[2] = {0, 0};
    CK(cudaMemcpyAsync(c, s->scratch + 8, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *evaluated = c[0];
    *skipped = c[1];
  });
}

RT_EXPORT void rteaal_sim_destroy(rteaal_sim* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  {
    std::lock_guard<std::mutex> g(s->design_mut->mu);
    s->design_mut->live_sims--;
  }
  delete s;
}

RT_EXPORT int rteaal_step(rteaal_sim* s, const rteaal_cycles* cycles, const rteaal_stimulus* stim,
                          const rteaal_probes* probes, uint32_t flags, void* stream);

RT_EXPORT int rteaal_sim_autotune(rteaal_sim* s, uint32_t cycles_per_trial, uint32_t kernel_mask,
                                  rteaal_tune_trial* trials, uint32_t max_trials, uint32_t* n_trials,
                                  void* stream) {
  return guarded([&] {
    require(s, "rteaal_sim_autotune: null sim");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(s->design->device));
    sync_sim(s, st);
    if (!cycles_per_trial) cycles_per_trial = 1;
    if (!kernel_mask)
      kernel_mask = s->n_pad >= 64 ? ((1u << RTEAAL_KERNEL_TILE) | (1u << RTEAAL_KERNEL_GRID) |
                                      (1u << RTEAAL_KERNEL_STREAM))
                                   : ((1u << RTEAAL_KERNEL_LAYER) | (1u << RTEAAL_KERNEL_GRID) |
                                      (1u << RTEAAL_KERNEL_CLUSTER) | (1u << RTEAAL_KERNEL_FLOW));
    const Lowered& L = s->design->L;
    const size_t np = s->n_pad;
    const size_t b_state = np * L.lane_bytes, b_mem = np * 8 * L.mem_words_total,
                 b_xs = np * 8 * L.in_width.size();
    // device snapshot of everything a trial can change
    char* snap = static_cast<char*>(s->alloc.alloc(b_state + b_mem + b_xs + 256));
    struct Free {
      rteaal_sim* s; void* p; size_t n;
      ~Free() { s->alloc.free(p, n); }
    } guard{s, snap, b_state + b_mem + b_xs + 256};
    CK(cudaMemcpyAsync(snap, s->state, b_state, cudaMemcpyDeviceToDevice, st));
    if (b_mem) CK(cudaMemcpyAsync(snap + b_state, s->mem, b_mem, cudaMemcpyDeviceToDevice, st));
    if (b_xs) CK(cudaMemcpyAsync(snap + b_state + b_mem, s->xs, b_xs, cudaMemcpyDeviceToDevice, st));

    struct Cand { int kernel; uint32_t T, threads, U, V; };
    std::vector<Cand> cands;
    struct CandX { int kernel; uint32_t T, threads, U, V, ctas; };
    std::vector<CandX> candx;
    if (kernel_mask & (1u << RTEAAL_KERNEL_TILE))
      for (uint32_t T : {8u, 16u, 32u, 64u})
        if (T <= np && np % T == 0)
          for (const Variant& v : all_variants())
            if (v.V >= 2 && T % (uint32_t)v.V == 0)
              candx.push_back({RTEAAL_KERNEL_TILE, T, (uint32_t)v.maxt, (uint32_t)v.U, (uint32_t)v.V, (uint32_t)v.minb});
    if (kernel_mask & (1u << RTEAAL_KERNEL_GRID))
      for (const Variant& v : all_variants())
        if (v.V >= 2 && np % (uint32_t)v.V == 0)
          candx.push_back({RTEAAL_KERNEL_GRID, 0, (uint32_t)v.maxt, (uint32_t)v.U, (uint32_t)v.V, (uint32_t)v.minb});
    if (kernel_mask & (1u << RTEAAL_KERNEL_LAYER))
      for (uint32_t V : {2u, 4u})
        for (uint32_t U : {1u, 2u, 4u}) cands.push_back({RTEAAL_KERNEL_LAYER, 0, 256, U, V});
    if (kernel_mask & (1u << RTEAAL_KERNEL_LAYER_GRAPH))
      for (uint32_t U : {2u, 4u}) cands.push_back({RTEAAL_KERNEL_LAYER_GRAPH, 0, 256, U, 0});
    if ((kernel_mask & (1u << RTEAAL_KERNEL_STREAM)) && np % 128 == 0)
      cands.push_back({RTEAAL_KERNEL_STREAM, 0, 0, 1, 0});
    if (kernel_mask & (1u << RTEAAL_KERNEL_CLUSTER)) {  // ctas: CTAs per cluster; U = 2 marks resident state
      const ClusterVariantTable ct = variants_cluster();
      for (size_t i = 0; i < ct.n; i++) {
        const ClusterVariant& cv = ct.v[i];
        if (cv.resident && np > 64) continue;
        for (uint32_t T : {np <= 256 ? (uint32_t)np : 256u, np <= 128 ? (uint32_t)np : 128u}) {
          if (np % T || T % (uint32_t)cv.V || (cv.resident && T != np)) continue;
          for (uint32_t cs : {16u, 8u, 4u})
            candx.push_back({RTEAAL_KERNEL_CLUSTER, T, (uint32_t)cv.maxt, cv.resident ? 2u : 1u, (uint32_t)cv.V, cs});
          if (T == np) break;
        }
      }
    }
    if (kernel_mask & (1u << RTEAAL_KERNEL_FLOW)) {
      const FlowVariantTable ft = variants_flow();
      for (size_t i = 0; i < ft.n; i++)  // T: items per warp
        for (uint32_t kw : {8u, 32u}) cands.push_back({RTEAAL_KERNEL_FLOW, kw, (uint32_t)ft.v[i].maxt, 1, 1});
    }
    for (const Cand& c : cands) candx.push_back({c.kernel, c.T, c.threads, c.U, c.V, 0});

    const int saved[6] = {s->kernel, (int)s->tile_lanes, (int)s->threads, (int)s->ctas_per_sm, (int)s->unroll,
                          s->V};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    rteaal_cycles cyc{cycles_per_trial, nullptr};
    rteaal_stimulus stim{L.in_width.empty() ? RTEAAL_STIM_HOLD : RTEAAL_STIM_XORSHIFT, nullptr, 0};
    float best = 1e30f;
    CandX best_c{saved[0], (uint32_t)saved[1], (uint32_t)saved[2], (uint32_t)saved[4], (uint32_t)saved[5],
                 (uint32_t)saved[3]};
    uint32_t best_ctas = (uint32_t)saved[3];
    uint32_t nt = 0;
    for (const CandX& c : candx) {
      try {
        const bool cl = c.kernel == RTEAAL_KERNEL_CLUSTER;
        configure(s, c.kernel, c.T, c.threads, cl ? 0 : c.ctas, cl ? 1 : c.U, c.V, cl ? c.ctas : 0,
                  cl ? (c.U == 2 ? 1 : -1) : 0);
      } catch (const Error&) {
        continue;  // not compiled / not resident
      }
      if (rteaal_step(s, &cyc, &stim, nullptr, 0, st) != RTEAAL_OK) { last_error().clear(); continue; }
      CK(cudaEventRecord(e0, st));
      if (rteaal_step(s, &cyc, &stim, nullptr, 0, st) != RTEAAL_OK) { last_error().clear(); continue; }
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      try { sync_sim(s, st); } catch (const Error&) { continue; }
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (trials && nt < max_trials)
        trials[nt] = rteaal_tune_trial{s->kernel, s->tile_lanes, s->threads,
                                       s->kernel == RTEAAL_KERNEL_CLUSTER ? s->cluster_ctas : s->ctas_per_sm,
                                       s->unroll, s->grid, (uint32_t)s->V, ms};
      nt++;
      if (ms < best) {
        best = ms;
        best_c = c;
        best_ctas = c.ctas ? c.ctas : s->kernel == RTEAAL_KERNEL_CLUSTER ? s->cluster_ctas
                                                                        : s->ctas_per_sm;  // selects it again
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_trials) *n_trials = nt;
    const bool best_cl = best_c.kernel == RTEAAL_KERNEL_CLUSTER;
    configure(s, best_c.kernel, best_c.T, best_c.threads, best_cl ? 0 : best_ctas, best_cl ? 1 : best_c.U,
              best_c.V, best_cl ? best_ctas : 0, best_cl ? (best_c.U == 2 ? 1 : -1) : 0);
    s->act_force = true;  // restored below; stamps of the trials are stale
    CK(cudaMemcpyAsync(s->state, snap, b_state, cudaMemcpyDeviceToDevice, st));
    if (b_mem) CK(cudaMemcpyAsync(s->mem, snap + b_state, b_mem, cudaMemcpyDeviceToDevice, st));
    if (b_xs) CK(cudaMemcpyAsync(s->xs, snap + b_state + b_mem, b_xs, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
  });
}

RT_EXPORT int rteaal_step(rteaal_sim* s, const rteaal_cycles* cycles, const rteaal_stimulus* stim,
                          const rteaal_probes* probes, uint32_t flags, void* stream) {
  return guarded([&] {
    require(s && cycles && stim, "rteaal_step: null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(s->design->device));
    check_pending(s);
    const rteaal_design* D = s->design;
    const Lowered& L = D->L;
    const size_t np = s->n_pad;
    require(stim->mode >= RTEAAL_STIM_HOLD && stim->mode <= RTEAAL_STIM_BUFFER, "rteaal_step: bad stimulus mode");
    require(stim->mode != RTEAAL_STIM_BUFFER || stim->values, "rteaal_step: BUFFER stimulus without values");

    DSim ds = dsim(s);
    ds.reset = (flags & RTEAAL_STEP_RESET) ? 1 : 0;
    ds.stim_mode = L.in_width.empty() ? 0 : stim->mode;

    // per-lane cycle budgets
    uint64_t max_cyc = 0;
    std::vector<uint32_t> hb;
    if (cycles->per_instance) {
      hb.assign(np, 0);
      for (uint32_t u = 0; u < s->n_user; u++) {
        hb[s->h_lane_of_user[u]] = cycles->per_instance[u];
        max_cyc = std::max<uint64_t>(max_cyc, cycles->per_instance[u]);
      }
      CK(cudaMemcpyAsync(s->budget, hb.data(), np * 4, cudaMemcpyHostToDevice, st));
      ds.budget = s->budget;
    } else {
      require(cycles->uniform <= 0xFFFFFFFFull, "rteaal_step: at most 2^32-1 cycles per call");
      max_cyc = cycles->uniform;
      ds.uniform = (uint32_t)max_cyc;
    }
    if (max_cyc == 0) return;
    if (cycles->reset_per_instance) {
      std::vector<uint32_t> hr(np, 0);
      for (uint32_t u = 0; u < s->n_user; u++) hr[s->h_lane_of_user[u]] = cycles->reset_per_instance[u];
      CK(cudaMemcpyAsync(s->reset_lane, hr.data(), np * 4, cudaMemcpyHostToDevice, st));
      ds.reset_lane = s->reset_lane;
    }

    // stimulus and probe buffers (host ones go through one device staging buffer)
    const size_t stim_host_bytes = (ds.stim_mode == RTEAAL_STIM_BUFFER && stim->values_on_host)
                                       ? (size_t)max_cyc * L.in_width.size() * s->n_user * 8 : 0;
    int probe_mode = RTEAAL_PROBE_LAST;
    size_t probe_bytes = 0;
    const bool probing = probes && probes->n;
    if (probing) {
      require(probes->signals && probes->out, "rteaal_step: probes without signals / out");
      probe_mode = probes->mode;
      require(probe_mode == RTEAAL_PROBE_LAST || probe_mode == RTEAAL_PROBE_EVERY ||
                  probe_mode == RTEAAL_PROBE_CHANGES,
              "rteaal_step: bad probe mode");
      if (probe_mode == RTEAAL_PROBE_CHANGES) {
        require(probes->count != nullptr, "rteaal_step: CHANGES probes need a count pointer");
        probe_bytes = (size_t)probes->capacity * sizeof(rteaal_change);
      } else {
        probe_bytes = (probe_mode == RTEAAL_PROBE_EVERY ? (size_t)max_cyc : 1) * probes->n * s->n_user * 8;
      }
    }
    const bool probe_host = probing && probes->out_on_host;
    ensure_staging(s, stim_host_bytes + (probe_host ? probe_bytes : 0));
    if (ds.stim_mode == RTEAAL_STIM_BUFFER) {
      if (stim_host_bytes) {
        CK(cudaMemcpyAsync(s->staging, stim->values, stim_host_bytes, cudaMemcpyHostToDevice, st));
        ds.stim = s->staging;
      } else {
        ds.stim = stim->values;
      }
    }
    uint64_t* probe_dev = nullptr;
    if (probing) {
      std::vector<uint32_t> slots(probes->n);
      for (uint32_t p = 0; p < probes->n; p++) {
        require(probes->signals[p] < D->nl.n_signals(), "rteaal_step: probe signal out of range");
        require(D->slot_of(probes->signals[p]) != 0xFFFFFFFFu,
                "rteaal_step: probed signal was fused away (operator fusion is enabled)");
        slots[p] = L.slot_ref[D->slot_of(probes->signals[p])];
      }
      ensure_probe_slots(s, slots.size());
      CK(cudaMemcpyAsync(s->probe_slots, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice, st));
      probe_dev = probe_host ? s->staging + stim_host_bytes / 8 : probes->out;
      if (probe_mode == RTEAAL_PROBE_EVERY || probe_mode == RTEAAL_PROBE_CHANGES) {
        ds.probe_slot = s->probe_slots;
        ds.n_probe = probes->n;
        ds.probe_out = probe_dev;
      }
      if (probe_mode == RTEAAL_PROBE_CHANGES) {
        // previous values = the probes' values as the step begins, lane order
        const size_t need = (size_t)probes->n * np * 8;
        if (s->probe_prev_bytes < need) {
          s->probe_prev = static_cast<uint64_t*>(s->get(need));
          s->probe_prev_bytes = need;
        }
        const uint32_t blocks = (uint32_t)std::min<size_t>((probes->n * np + 255) / 256, 4096);
        k_gather_ref<<<blocks, 256, 0, st>>>(s->state, s->n_pad, s->probe_slots, probes->n, nullptr, 0,
                                             s->n_pad, s->probe_prev);
        CK(cudaGetLastError());
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(s->scratch + 16);
        CK(cudaMemsetAsync(cnt, 0, 8, st));
        ds.probe_changes = 1;
        ds.probe_prev = s->probe_prev;
        ds.change_count = cnt;
        ds.change_cap = probes->capacity;
      }
    }

    const uint32_t U = s->unroll;
    // lanes this step visits (STREAM: whole chunks; the others: whole warps)
    const uint32_t span = live_span(s, hb, s->kernel == RTEAAL_KERNEL_STREAM ? s->stream_chunk
                                           : s->kernel == RTEAAL_KERNEL_SPECIALIZED ? kSpecThreads
                                           : s->kernel == RTEAAL_KERNEL_CLUSTER ? s->tile_lanes
                                           : s->kernel == RTEAAL_KERNEL_FLOW ? 1u
                                           : 32u * (uint32_t)s->V);
    s->last_span = span;
    if (s->kernel == RTEAAL_KERNEL_LAYER) {
      for (uint64_t c = 0; c < max_cyc; c++) {
        if (s->V == 4) launch_layer_cycle<4>(s, D->dd, ds, (uint32_t)c, nullptr, st, D->n_sms, span);
        else if (s->V == 2) launch_layer_cycle<2>(s, D->dd, ds, (uint32_t)c, nullptr, st, D->n_sms, span);
        else launch_layer_cycle<1>(s, D->dd, ds, (uint32_t)c, nullptr, st, D->n_sms, span);
      }
      CK(cudaGetLastError());
    } else if (s->kernel == RTEAAL_KERNEL_LAYER_GRAPH) {
      uint32_t* cyc_dev = s->scratch + 4;
      CK(cudaMemsetAsync(cyc_dev, 0, 4, st));
      cudaStream_t cap;
      CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      try {
        CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (s->V == 4) launch_layer_cycle<4>(s, D->dd, ds, 0u, cyc_dev, cap, D->n_sms, span);
        else if (s->V == 2) launch_layer_cycle<2>(s, D->dd, ds, 0u, cyc_dev, cap, D->n_sms, span);
        else launch_layer_cycle<1>(s, D->dd, ds, 0u, cyc_dev, cap, D->n_sms, span);
        k_tick<<<1, 1, 0, cap>>>(cyc_dev);
        CK(cudaStreamEndCapture(cap, &g));
        CK(cudaGraphInstantiate(&ge, g, 0));
        for (uint64_t c = 0; c < max_cyc; c++) CK(cudaGraphLaunch(ge, st));
      } catch (...) {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        throw;
      }
      // the exec graph may be destroyed while launches are pending (CUDA keeps them alive)
      cudaGraphExecDestroy(ge);
      cudaGraphDestroy(g);
      cudaStreamDestroy(cap);
    } else if (s->kernel == RTEAAL_KERNEL_SPECIALIZED) {
      require(max_cyc <= 0xFFFFFFFFull, "rteaal_step: too many cycles");
      if (probing && probe_mode != RTEAAL_PROBE_LAST)
        throw Error(RTEAAL_E_UNSUPPORTED, "design-specialised kernel: probes in LAST mode only");
      uint8_t* a_st = s->state;
      uint64_t* a_mem = s->mem;
      uint64_t* a_xs = s->xs;
      const uint64_t* a_stim = ds.stim;
      const uint32_t* a_budget = ds.budget;
      const uint32_t* a_rl = ds.reset_lane;
      const uint32_t* a_uol = ds.user_of_lane;
      uint32_t a_np = s->n_pad, a_nu = s->n_user, a_uni = ds.uniform;
      int a_mode = ds.stim_mode, a_reset = ds.reset;
      void* args[] = {&a_st, &a_mem, &a_xs, &a_stim, &a_budget, &a_rl, &a_uol, &a_np, &a_nu, &a_uni, &a_mode, &a_reset};
      CK(cudaLaunchKernel((const void*)D->spec_kernel, dim3((span + kSpecThreads - 1) / kSpecThreads),
                          dim3(kSpecThreads), args, 0, st));
      CK(cudaGetLastError());
    } else if (s->kernel == RTEAAL_KERNEL_CLUSTER && s->resident) {
      require(max_cyc <= 0xFFFFFFFFull, "rteaal_step: too many cycles");
      ResidentArgs ra{};
      ra.ncyc = (uint32_t)max_cyc;
      ra.bytes = (uint32_t)(np * L.lane_bytes);
      ra.slice = make_fastdiv(s->res_slice);
      ra.tpo = make_fastdiv((uint32_t)np);
      ra.stage_cap = s->stage_cap;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = s->cluster_ctas;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(s->cluster_ctas);
      cfg.blockDim = dim3(s->threads);
      cfg.dynamicSmemBytes = s->res_smem;
      cfg.stream = st;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      void* args[] = {(void*)&D->dd, (void*)&ds, (void*)&ra};
      s->last_grid = s->cluster_ctas;
      CK(cudaLaunchKernelExC(&cfg, s->cluster_fn, args));
      CK(cudaGetLastError());
    } else if (s->kernel == RTEAAL_KERNEL_CLUSTER) {
      require(max_cyc <= 0xFFFFFFFFull, "rteaal_step: too many cycles");
      const uint32_t T = s->tile_lanes;
      const uint32_t n_tiles = span / T;
      ClusterArgs ca{};
      ca.tile_lanes = T;
      ca.n_tiles = n_tiles;
      ca.tpo = make_fastdiv(T / (uint32_t)s->V);
      ca.stage_cap = s->stage_cap;
      if (cycles->per_instance) {
        std::vector<uint32_t> tc(n_tiles, 0);
        for (uint32_t t = 0; t < n_tiles; t++)
          for (uint32_t l = 0; l < T; l++) tc[t] = std::max(tc[t], hb[(size_t)t * T + l]);
        CK(cudaMemcpyAsync(s->tile_cycles, tc.data(), n_tiles * 4, cudaMemcpyHostToDevice, st));
        ca.tile_cycles = s->tile_cycles;
      }
      require(s->cluster_fn != nullptr, "rteaal_step: no cluster variant for this configuration");
      const uint32_t n_cl = std::max<uint32_t>(1, std::min(s->n_clusters, n_tiles));
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = s->cluster_ctas;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(n_cl * s->cluster_ctas);
      cfg.blockDim = dim3(s->threads);
      cfg.dynamicSmemBytes = cluster_table_smem(s->stage_cap, D->dd.n_layers);
      cfg.stream = st;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      void* args[] = {(void*)&D->dd, (void*)&ds, (void*)&ca};
      s->last_grid = n_cl * s->cluster_ctas;
      CK(cudaLaunchKernelExC(&cfg, s->cluster_fn, args));
      CK(cudaGetLastError());
    } else if (s->kernel == RTEAAL_KERNEL_TILE) {
      require(max_cyc <= 0xFFFFFFFFull, "rteaal_step: too many cycles");
      const uint32_t T = s->tile_lanes;
      const uint32_t n_tiles = (uint32_t)(np / T);
      TileArgs ta{};
      ta.counter = s->scratch + 1;
      ta.n_tiles = n_tiles;
      ta.tile_lanes = T;
      ta.tpo = make_fastdiv(T / s->V);
      if (cycles->per_instance) {
        std::vector<uint32_t> tc(n_tiles, 0), order(n_tiles);
        for (uint32_t t = 0; t < n_tiles; t++)
          for (uint32_t l = 0; l < T; l++) tc[t] = std::max(tc[t], hb[(size_t)t * T + l]);
        std::iota(order.begin(), order.end(), 0u);
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return tc[a] > tc[b]; });
        CK(cudaMemcpyAsync(s->tile_cycles, tc.data(), n_tiles * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(s->tile_order, order.data(), n_tiles * 4, cudaMemcpyHostToDevice, st));
        ta.tile_cycles = s->tile_cycles;
        ta.order = s->tile_order;
      }
      CK(cudaMemsetAsync(ta.counter, 0, 4, st));
      const uint32_t grid = std::min<uint32_t>(s->grid, n_tiles);
      const Variant* v = find_variant(s->V, U, s->threads);
      require(v != nullptr, "rteaal_step: no kernel variant for this configuration");
      void* args[] = {(void*)&D->dd, (void*)&ds, (void*)&ta};
      CK(cudaLaunchKernel(v->tile, dim3(grid), dim3(s->threads), args, 0, st));
      CK(cudaGetLastError());
    } else if (s->kernel == RTEAAL_KERNEL_STREAM) {
      require(max_cyc <= 0xFFFFFFFFull, "rteaal_step: too many cycles");
      GridArgs ga{};
      ga.count = reinterpret_cast<unsigned long long*>(s->scratch + 2);
      ga.expected = s->grid + s->barrier_extra;
      ga.timeout_ns = s->barrier_timeout_ns;
      ga.ncyc = (uint32_t)max_cyc;
      ga.tpo = make_fastdiv(span / STREAM_V);
      const uint32_t half = s->stream_chunk / 128u;
      StreamArgs sa{half, span / s->stream_chunk};
      CK(cudaMemsetAsync(s->scratch, 0, 16, st));
      void* args[] = {(void*)&D->dd, (void*)&ds, (void*)&ga, (void*)&sa};
      cudaError_t e = cudaLaunchCooperativeKernel(half == 2 ? (const void*)k_stream<2> : (const void*)k_stream<1>,
                                                  dim3(s->grid), dim3(s->threads), args, stream_smem_bytes(), st);
      if (e == cudaErrorCooperativeLaunchTooLarge)
        throw Error(RTEAAL_E_UNSUPPORTED, "cooperative grid does not fit on the device");
      CK(e);
      CK(cudaMemcpyAsync(s->err_host, s->scratch, 4, cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(s->done, st));
      s->pending = true;
    } else if (s->kernel == RTEAAL_KERNEL_FLOW) {
      require(max_cyc <= 0xFFFFFFFFull, "rteaal_step: too many cycles");
      const size_t mirror_bytes = (size_t)L.n_slots * s->n_pad * 16;
      if (!s->flow_mirror) {
        s->flow_mirror = static_cast<unsigned long long*>(s->get(std::max<size_t>(mirror_bytes, 16)));
        CK(cudaMemsetAsync(s->flow_mirror, 0, mirror_bytes, st));
        s->flow_epoch = 0;
        std::vector<uint32_t> fop, fext, fpool;
        flow_tables(L, fop, fext, fpool);
        if (fop.empty()) fop.assign(8, 0u);
        if (fext.empty()) fext.push_back(0u);
        if (fpool.empty()) fpool.assign(2, 0u);
        s->flow_op = static_cast<uint4*>(s->get(fop.size() * 4));      // 2 uint4 per op
        s->flow_ext = static_cast<uint32_t*>(s->get(fext.size() * 4));
        s->flow_pool = static_cast<uint2*>(s->get(fpool.size() * 4));  // 1 uint2 per row
        CK(cudaMemcpyAsync(s->flow_op, fop.data(), fop.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(s->flow_ext, fext.data(), fext.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(s->flow_pool, fpool.data(), fpool.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));  // the host vectors go out of scope
      }
      if ((uint64_t)s->flow_epoch + max_cyc >= 0xFFFFFFFFull) {  // stamps would wrap: start over
        CK(cudaMemsetAsync(s->flow_mirror, 0, mirror_bytes, st));
        s->flow_epoch = 0;
      }
      // threads for the widest phase: a layer at flow_kw items per warp, the edge
      // or the stimulus at one item per thread
      const uint64_t widest = std::max<uint64_t>(
          {(uint64_t)L.max_layer_ops * 32 / s->flow_kw, L.reg_src.size() + (L.mem_info.size() / 4 - 1),
           (uint64_t)L.in_width.size(), 1});
      const uint32_t grid = (uint32_t)std::max<uint64_t>(
          1, std::min<uint64_t>(s->grid, (widest * span + s->threads - 1) / s->threads));
      GridArgs ga{};
      ga.count = reinterpret_cast<unsigned long long*>(s->scratch + 2);
      ga.expected = grid + s->barrier_extra;
      ga.timeout_ns = 2 * s->barrier_timeout_ns;
      ga.ncyc = (uint32_t)max_cyc;
      ga.tpo = make_fastdiv(span);
      FlowArgs fa{};
      fa.timeout_ns = s->barrier_timeout_ns;
      fa.mirror = s->flow_mirror;
      fa.fop = s->flow_op;
      fa.fext = s->flow_ext;
      fa.fpool = s->flow_pool;
      fa.n_in = (uint32_t)D->L.in_ref.size();
      fa.n_reg = (uint32_t)D->L.reg_ref.size();
      fa.n_const = (uint32_t)D->L.const_ref.size();
      fa.epoch = s->flow_epoch;
      fa.skew = s->flow_skew;
      fa.span = make_fastdiv(span);
      const size_t off_bytes = (size_t)D->L.layer_off.size() * 4;
      fa.off_in_smem = off_bytes <= kFlowOffSmem;
      fa.kw = s->flow_kw;
      CK(cudaMemsetAsync(s->scratch, 0, 16, st));
      void* args[] = {(void*)&D->dd, (void*)&ds, (void*)&ga, (void*)&fa};
      s->last_grid = grid;
      cudaError_t e = cudaLaunchCooperativeKernel(s->flow_fn, dim3(grid), dim3(s->threads), args,
                                                  fa.off_in_smem ? off_bytes : 0, st);
      if (e == cudaErrorCooperativeLaunchTooLarge)
        throw Error(RTEAAL_E_UNSUPPORTED, "cooperative grid does not fit on the device");
      CK(e);
      s->flow_epoch += (uint32_t)max_cyc;
      CK(cudaMemcpyAsync(s->err_host, s->scratch, 4, cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(s->done, st));
      s->pending = true;
    } else {  // GRID
      require(max_cyc <= 0xFFFFFFFFull, "rteaal_step: too many cycles");
      const uint32_t grid = grid_for_span(s, span, (uint32_t)s->V);
      GridArgs ga{};
      ga.count = reinterpret_cast<unsigned long long*>(s->scratch + 2);
      ga.expected = grid + s->barrier_extra;
      ga.timeout_ns = s->barrier_timeout_ns;
      ga.ncyc = (uint32_t)max_cyc;
      ga.tpo = make_fastdiv(span / (uint32_t)s->V);
      ga.stage_cap = s->activity ? 0u : s->stage_cap;
      CK(cudaMemsetAsync(s->scratch, 0, 16, st));
      const void* fn = nullptr;
      if (s->activity) {
        const ActVariant* av = find_act_variant(s->V, s->threads);
        require(av != nullptr, "rteaal_step: no activity-aware variant for this configuration");
        fn = av->grid;
        // uneven budgets leave some lanes' last edge unseen by the next step's
        // first cycle, which therefore evaluates everything
        bool uneven = false;
        if (cycles->per_instance)
          for (uint32_t u = 0; u < s->n_user && !uneven; u++) uneven = cycles->per_instance[u] != max_cyc;
        s->act_g += max_cyc;
        s->act_force = uneven;
      } else {
        const Variant* v = find_variant(s->V, U, s->threads);
        require(v != nullptr, "rteaal_step: no kernel variant for this configuration");
        fn = v->grid;
      }
      void* args[] = {(void*)&D->dd, (void*)&ds, (void*)&ga};
      s->last_grid = grid;
      cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(s->threads), args,
                                                  (size_t)ga.stage_cap * kStageBytes, st);
      if (e == cudaErrorCooperativeLaunchTooLarge)
        throw Error(RTEAAL_E_UNSUPPORTED, "cooperative grid does not fit on the device");
      CK(e);
      CK(cudaMemcpyAsync(s->err_host, s->scratch, 4, cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(s->done, st));
      s->pending = true;
    }

    if (probing && probe_mode == RTEAAL_PROBE_LAST) {
      const size_t total = (size_t)probes->n * s->n_user;
      const uint32_t blocks = (uint32_t)std::min<size_t>((total + 255) / 256, 4096);
      k_gather_ref<<<blocks, 256, 0, st>>>(s->state, s->n_pad, s->probe_slots, probes->n, s->lane_of_user,
                                           0, s->n_user, probe_dev);
      CK(cudaGetLastError());
    }
    if (probing && probe_mode == RTEAAL_PROBE_CHANGES) {
      uint64_t count = 0;
      CK(cudaMemcpyAsync(&count, s->scratch + 16, 8, cudaMemcpyDeviceToHost, st));
      sync_sim(s, st);
      *probes->count = count;
      if (probe_host && count)
        CK(cudaMemcpy(probes->out, probe_dev, (size_t)std::min<uint64_t>(count, probes->capacity) *
                                                  sizeof(rteaal_change), cudaMemcpyDeviceToHost));
    } else if (probe_host) {
      CK(cudaMemcpyAsync(probes->out, probe_dev, probe_bytes, cudaMemcpyDeviceToHost, st));
      sync_sim(s, st);
    } else if (stim_host_bytes) {
      // the caller may reuse its host buffer once we return
      sync_sim(s, st);
    }
  });
}

RT_EXPORT int rteaal_sim_reset_lanes(rteaal_sim* s, uint32_t inst0, uint32_t n_inst, const uint64_t* seed,
                                     void* stream) {
  return guarded([&] {
    require(s, "rteaal_sim_reset_lanes: null sim");
    require((uint64_t)inst0 + n_inst <= s->n_user, "rteaal_sim_reset_lanes: instance range out of bounds");
    if (n_inst == 0) return;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(s->design->device));
    check_pending(s);
    const rteaal_design* D = s->design;
    const Lowered& L = D->L;
    const uint32_t ni = (uint32_t)L.in_width.size();
    const uint64_t* xs_in = nullptr;
    if (seed && ni) {
      ensure_staging(s, (size_t)ni * n_inst * 8);
      CK(cudaMemcpyAsync(s->staging, seed, (size_t)ni * n_inst * 8, cudaMemcpyHostToDevice, st));
      xs_in = s->staging;
    }
    const size_t total = ((size_t)L.n_slots + L.mem_words_total + ni) * n_inst;
    const uint32_t blocks = (uint32_t)std::min<size_t>((total + 255) / 256, (size_t)D->n_sms * 32);
    s->act_force = true;
    k_reset_lanes<<<blocks, 256, 0, st>>>(s->state, s->mem, s->xs, s->n_pad, D->d_slot_ref, L.n_slots, L.const_base,
                                          (uint32_t)L.const_value.size(), D->d_const_value, L.mem_words_total,
                                          ni, xs_in, s->lane_of_user, inst0, n_inst);
    CK(cudaGetLastError());
    if (xs_in) CK(cudaStreamSynchronize(st));  // the staging buffer may be reused by the next call
  });
}

RT_EXPORT int rteaal_sync(rteaal_sim* s, void* stream) {
  return guarded([&] {
    require(s, "rteaal_sync: null sim");
    sync_sim(s, static_cast<cudaStream_t>(stream));
  });
}

namespace {

enum class Region { STATE, MEM, XS };

void transfer(rteaal_sim* s, Region region, const uint32_t* signals, uint32_t n, uint32_t inst0, uint32_t n_inst,
              uint64_t* out, const uint64_t* in, cudaStream_t st) {
  require(s, "null sim");
  if (in) s->act_force = true;  // written values carry no change stamps
  require(out || in, "null host buffer");
  require((uint64_t)inst0 + n_inst <= s->n_user, "instance range out of bounds");
  CK(cudaSetDevice(s->design->device));
  const Lowered& L = s->design->L;
  std::vector<uint32_t> rows;
  std::vector<uint64_t> masks;
  uint64_t* base = nullptr;
  uint32_t n_rows = n;
  if (region == Region::STATE) {
    require(signals || n == 0, "null signal list");
    rows.resize(n);
    masks.resize(n);
    const uint32_t nsig = s->design->nl.n_signals();
    for (uint32_t i = 0; i < n; i++) {
      require(signals[i] < nsig, "signal id out of range");
      require(s->design->slot_of(signals[i]) != 0xFFFFFFFFu, "signal was fused away (operator fusion is enabled)");
      rows[i] = L.slot_ref[s->design->slot_of(signals[i])];
      // width of the signal (writes are masked like every stored value)
      const Netlist& nl = s->design->nl;
      uint32_t sig = signals[i], w;
      if (sig < nl.ni) w = nl.in_w[sig];
      else if (sig < nl.ni + nl.nr) w = nl.reg_w[sig - nl.ni];
      else if (sig < nl.op_base()) w = nl.const_w[sig - nl.ni - nl.nr];
      else w = nl.width[sig - nl.op_base()];
      masks[i] = ~0ull >> (64 - w);
    }
  } else if (region == Region::MEM) {
    base = s->mem;
    n_rows = (uint32_t)L.mem_words_total;
  } else {
    base = s->xs;
    n_rows = (uint32_t)L.in_width.size();
  }
  const size_t total = (size_t)n_rows * n_inst;
  if (total == 0) return;
  sync_sim(s, st);
  void* tmp = s->alloc.alloc(total * 8 + rows.size() * 4 + masks.size() * 8 + 64);
  try {
    uint64_t* buf = static_cast<uint64_t*>(tmp);
    uint64_t* dmask = masks.empty() ? nullptr : buf + total;
    uint32_t* drows = rows.empty() ? nullptr : reinterpret_cast<uint32_t*>(buf + total + masks.size());
    if (drows) CK(cudaMemcpyAsync(drows, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, st));
    if (dmask) CK(cudaMemcpyAsync(dmask, masks.data(), masks.size() * 8, cudaMemcpyHostToDevice, st));
    const uint32_t blocks = (uint32_t)std::min<size_t>((total + 255) / 256, 8192);
    const bool compact = region == Region::STATE;
    if (out) {
      if (compact)
        k_gather_ref<<<blocks, 256, 0, st>>>(s->state, s->n_pad, drows, n_rows, s->lane_of_user, inst0, n_inst, buf);
      else
        k_gather<<<blocks, 256, 0, st>>>(base, s->n_pad, drows, n_rows, s->lane_of_user, inst0, n_inst, buf);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(out, buf, total * 8, cudaMemcpyDeviceToHost, st));
    } else {
      CK(cudaMemcpyAsync(buf, in, total * 8, cudaMemcpyHostToDevice, st));
      if (compact)
        k_scatter_ref<<<blocks, 256, 0, st>>>(s->state, s->n_pad, drows, n_rows, s->lane_of_user, inst0, n_inst,
                                              buf, dmask);
      else
        k_scatter<<<blocks, 256, 0, st>>>(base, s->n_pad, drows, n_rows, s->lane_of_user, inst0, n_inst, buf,
                                          nullptr);
      CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(st));
  } catch (...) {
    s->alloc.free(tmp, total * 8 + rows.size() * 4 + masks.size() * 8 + 64);
    throw;
  }
  s->alloc.free(tmp, total * 8 + rows.size() * 4 + masks.size() * 8 + 64);
}

}  // namespace

RT_EXPORT int rteaal_state_read(rteaal_sim* s, const uint32_t* signals, uint32_t n, uint32_t inst0,
                                uint32_t n_inst, uint64_t* out, void* stream) {
  return guarded([&] { transfer(s, Region::STATE, signals, n, inst0, n_inst, out, nullptr, (cudaStream_t)stream); });
}

RT_EXPORT int rteaal_state_write(rteaal_sim* s, const uint32_t* signals, uint32_t n, uint32_t inst0,
                                 uint32_t n_inst, const uint64_t* in, void* stream) {
  return guarded([&] { transfer(s, Region::STATE, signals, n, inst0, n_inst, nullptr, in, (cudaStream_t)stream); });
}

RT_EXPORT int rteaal_mem_read(rteaal_sim* s, uint32_t inst0, uint32_t n_inst, uint64_t* out, void* stream) {
  return guarded([&] { transfer(s, Region::MEM, nullptr, 0, inst0, n_inst, out, nullptr, (cudaStream_t)stream); });
}

RT_EXPORT int rteaal_mem_write(rteaal_sim* s, uint32_t inst0, uint32_t n_inst, const uint64_t* in, void* stream) {
  return guarded([&] { transfer(s, Region::MEM, nullptr, 0, inst0, n_inst, nullptr, in, (cudaStream_t)stream); });
}

RT_EXPORT int rteaal_stim_state_read(rteaal_sim* s, uint32_t inst0, uint32_t n_inst, uint64_t* out, void* stream) {
  return guarded([&] { transfer(s, Region::XS, nullptr, 0, inst0, n_inst, out, nullptr, (cudaStream_t)stream); });
}

RT_EXPORT int rteaal_stim_state_write(rteaal_sim* s, uint32_t inst0, uint32_t n_inst, const uint64_t* in,
                                      void* stream) {
  return guarded([&] { transfer(s, Region::XS, nullptr, 0, inst0, n_inst, nullptr, in, (cudaStream_t)stream); });
}

// ================================================================== allocation-free step
//
// For callers that cannot allocate device memory themselves: everything the
// persistent grid kernel needs besides the caller's buffers (error word,
// barrier arrival count, per-lane cycle budgets) lives in one
// file-scope device array.  Every GPU that loads this library holds the array
// (RTEAAL_STATIC_MAX_LANES * 4 + 256 bytes) until the process exits.

static __device__ __align__(256) uint32_t g_static_scratch[64 + RTEAAL_STATIC_MAX_LANES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
uint32_t* g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once per
// device: host code only sees a host-side stand-in under that name).
uint32_t* static_scratch(int dev) {
  require(dev >= 0 && dev < kMaxDevices, "rteaal_step_static: device ordinal out of range");
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[dev] = static_cast<uint32_t*>(p);
  }
  return g_static_addr[dev];
}

}  // namespace

RT_EXPORT int rteaal_step_static(const rteaal_design* d, void* state, uint64_t* mem, uint64_t* xs,
                                 uint32_t n_lanes, const uint32_t* cycles, uint32_t uniform_cycles,
                                 int stim_mode, uint32_t flags, void* stream) {
  return guarded([&] {
    require(d && state, "rteaal_step_static: null design or state");
    require(n_lanes >= 1, "rteaal_step_static: n_lanes must be at least 1");
    if (n_lanes > RTEAAL_STATIC_MAX_LANES)
      throw Error(RTEAAL_E_INVALID, "rteaal_step_static: n_lanes " + std::to_string(n_lanes) +
                                        " exceeds the static scratch limit of " +
                                        std::to_string(RTEAAL_STATIC_MAX_LANES) + " lanes");
    require(stim_mode == RTEAAL_STIM_HOLD || stim_mode == RTEAAL_STIM_XORSHIFT,
            "rteaal_step_static: stimulus mode must be HOLD or XORSHIFT");
    const Lowered& L = d->L;
    require(mem || L.mem_words_total == 0, "rteaal_step_static: design has memories but mem is null");
    require(xs || stim_mode != RTEAAL_STIM_XORSHIFT || L.in_width.empty(),
            "rteaal_step_static: XORSHIFT stimulus needs xs");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(d->device));
    uint32_t* scratch = static_scratch(d->device);

    uint32_t max_cyc = uniform_cycles;
    if (cycles) {
      max_cyc = 0;
      for (uint32_t l = 0; l < n_lanes; l++) max_cyc = std::max(max_cyc, cycles[l]);
    }
    if (max_cyc == 0) return;
    const bool aligned = ((uintptr_t)state % 16 == 0) && ((uintptr_t)mem % 16 == 0) && ((uintptr_t)xs % 16 == 0);
    const int V = (n_lanes % 2 == 0 && aligned) ? 2 : 1;
    const uint32_t threads = 512;
    const Variant* v = find_variant(V, 1, threads);
    require(v != nullptr, "rteaal_step_static: no kernel variant");
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v->grid, (int)threads, 0));
    require(occ >= 1, "rteaal_step_static: kernel cannot be resident");
    const uint32_t grid = (uint32_t)occ * (uint32_t)d->n_sms;

    // the barrier and error words must start at zero; budgets are rewritten
    CK(cudaMemsetAsync(scratch, 0, 64 * sizeof(uint32_t), st));
    DSim ds{};
    ds.state = static_cast<uint8_t*>(state);
    ds.mem = mem;
    ds.xs = xs;
    ds.n_pad = n_lanes;
    ds.n_user = n_lanes;
    ds.stim_mode = L.in_width.empty() ? 0 : stim_mode;
    ds.reset = (flags & RTEAAL_STEP_RESET) ? 1 : 0;
    ds.err = scratch;
    if (cycles) {
      CK(cudaMemcpyAsync(scratch + 64, cycles, (size_t)n_lanes * 4, cudaMemcpyHostToDevice, st));
      ds.budget = scratch + 64;
    } else {
      ds.uniform = uniform_cycles;
    }
    GridArgs ga{};
    ga.count = reinterpret_cast<unsigned long long*>(scratch + 2);
    ga.expected = grid;
    ga.timeout_ns = 2000000000ull;
    // the same wait bound and test hook as the regular grid launch
    if (const char* e = getenv("RTEAAL_BARRIER_TIMEOUT_NS")) ga.timeout_ns = strtoull(e, nullptr, 10);
    if (const char* e = getenv("RTEAAL_TEST_WITHHOLD_ARRIVAL")) ga.expected += (uint32_t)atoi(e);
    ga.ncyc = max_cyc;
    ga.tpo = make_fastdiv(n_lanes / V);
    void* args[] = {(void*)&d->dd, (void*)&ds, (void*)&ga};
    cudaError_t e = cudaLaunchCooperativeKernel(v->grid, dim3(grid), dim3(threads), args, 0, st);
    if (e == cudaErrorCooperativeLaunchTooLarge)
      throw Error(RTEAAL_E_UNSUPPORTED, "cooperative grid does not fit on the device");
    CK(e);
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&err, scratch, sizeof(err), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err) throw Error(RTEAAL_E_TIMEOUT, "rteaal_step_static: a grid barrier wait timed out");
  });
}
