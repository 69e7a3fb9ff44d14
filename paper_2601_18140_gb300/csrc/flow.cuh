// flow.cuh -- the FLOW form: the layers of a cycle without barriers between them.
//
// For one instance, or a few, a layer is a few thousand items, and the barrier
// that separates two layers (Cascade 1's LI_{i+1} <- LO_i step) costs more than
// the layer's own work.  In this form a grid barrier is kept only around the
// stimulus and the clock edge.  Every row also has a pair of stamped words per
// lane (its value's low and high halves, each next to a stamp, one 16-byte
// store): an op writes its result there with the cycle's stamp, then to its
// compact row (which the clock edge, probes and state reads use); inputs,
// registers and constants are copied there after the stimulus and the edge.
// An item loads each operand's words with one branch-free 16-byte load, all
// of them before any is used, and waits until the operands that ops write in
// this cycle carry this cycle's stamp -- so a layer waits for exactly the
// results it reads, not for the whole layer below.
//
// Progress: every thread walks the layers in order, and an item waits only for
// items of lower layers, which their threads reach before this one (the same
// order) -- and every block is resident (cooperative launch), so every wait
// ends.  Each wait is still bounded by %globaltimer: after timeout_ns the thread
// sets error bit 8, every thread stops waiting once it sees the error word, and
// the kernel leaves at its next grid barrier.  The barriers of this form wait
// up to twice that bound, since a block may legitimately arrive one stamp wait
// late; a wait that gives up is thus reported as a stamp wait.
#pragma once
#include <cstddef>
#include <cstdint>

#include "flow_items.cuh"
#include "persistent.cuh"

namespace rteaal {

template <int MAXT>
__global__ void __launch_bounds__(MAXT) k_flow(DDesign d, DSim s, GridArgs g, FlowArgs f) {
  __shared__ int sh_ok;
  extern __shared__ uint32_t sm_off[];  // [n_layers + 1] layer offsets, when the launch gives room
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, T = gridDim.x * blockDim.x;
  const uint32_t* off = d.layer_off;
  if (f.off_in_smem) {
    for (uint32_t i = threadIdx.x; i <= d.n_layers; i += blockDim.x) sm_off[i] = __ldg(&d.layer_off[i]);
    __syncthreads();
    off = sm_off;
  }
#define RT_SPACE make_space<1>(f.span, 0u, t, T)
  // the rows no op writes, as they stand before the launch (registers and
  // inputs are refreshed again after the edge and the stimulus of each cycle)
  flow_refresh(s, f, RT_SPACE, 0u, f.n_in + f.n_reg + f.n_const);
  for (uint32_t c = 0; c < g.ncyc; c++) {
    stim_items<1>(d, s, RT_SPACE, c);
    flow_refresh(s, f, RT_SPACE, 0u, f.n_in);
    if (!grid_sync(g, s.err, &sh_ok)) return;
    flow_cycle(d, s, f, off, c, t, T, f.timeout_ns);  // a wait that gave up set the error word
    if (!grid_sync(g, s.err, &sh_ok)) return;
    commit_items<1>(d, s, RT_SPACE, c);
    flow_refresh(s, f, RT_SPACE, f.n_in, f.n_in + f.n_reg);
    if (!grid_sync(g, s.err, &sh_ok)) return;
    if (s.n_probe) {
      probe_items<1>(s, RT_SPACE, c);
      if (!grid_sync(g, s.err, &sh_ok)) return;
    }
  }
#undef RT_SPACE
}

struct FlowVariant {
  int maxt;
  const void* fn;
};
struct FlowVariantTable {
  const FlowVariant* v;
  size_t n;
};
#define RT_FLOW_VARIANT(T) {T, (const void*)k_flow<T>}
FlowVariantTable variants_flow();  // variants_flow.cu

}  // namespace rteaal
