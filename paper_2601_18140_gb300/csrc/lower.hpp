// lower.hpp -- netlist parsing and the netlist -> device-tensor lowering.
//
// The lowering realises the paper's compile flow (Sec. 6.1, Fig. "compiler"):
// levelisation by topological sort (Sec. 4.2), the OIM built per layer with
// operations of one type grouped together (the swizzled [I, N, S, O, R] format
// of the NU kernel, Sec. 5.2 / Fig. "opt-space:format"c), and identity
// elision by assigning every signal one global slot (Sec. 4.3, Sec. 6.1).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace rteaal {

enum Opcode : uint8_t {
  OP_COPY = 0, OP_AND, OP_OR, OP_XOR, OP_NOT, OP_ADD, OP_SUB, OP_MUL, OP_SHL, OP_SHR, OP_DSHL,
  OP_DSHR, OP_BITS, OP_CAT, OP_EQ, OP_NEQ, OP_LT, OP_LEQ, OP_GT, OP_GEQ, OP_MUX, OP_ANDR, OP_ORR,
  OP_XORR, OP_MEMRD, OP_MUXCHAIN, OP_COUNT
};

// ctl word of a lowered op: opcode (5 bits) | arity (2 bits, 1..3) << 5 |
// extended-operand flag << 7 | width (7 bits) << 8 | narrow flag << 15 |
// p0 << 16 | p1 << 24.  Narrow: the result and every operand fit 32 bits, so
// the op may be evaluated in 32-bit arithmetic (exact: the result is masked to
// at most 32 bits, and every opcode's low 32 bits depend only on the operands'
// low 32 bits or are 0 -- shifts by 32 or more, see the kernels).
constexpr uint32_t CTL_EXT = 1u << 7;
constexpr uint32_t CTL_NARROW = 1u << 15;
inline constexpr uint32_t ctl_width(uint32_t ctl) { return (ctl >> 8) & 127u; }

// Row reference: width class k (bytes per lane = 1 << k) in bits 30..31, the
// row's per-lane byte offset in bits 0..29.  Element (row, lane) of a state
// with n lanes lives at byte  offset * n + (lane << k).
constexpr uint32_t REF_OFF_MASK = (1u << 30) - 1u;
inline uint32_t width_class(uint32_t w) { return w <= 8 ? 0u : w <= 16 ? 1u : w <= 32 ? 2u : 3u; }

struct Netlist {
  uint32_t ni = 0, nr = 0, nc = 0, no = 0, nm = 0, nw = 0, na = 0;
  std::vector<uint64_t> reg_init, const_value;
  std::vector<uint32_t> reg_d, argoff, args, mem_words, wport;  // wport: 4 per port
  std::vector<uint8_t> in_w, reg_w, const_w, code, width, p0, p1, mem_w;
  uint32_t nd = 0;                                  // clock domains (0: one clock)
  std::vector<uint32_t> dom_period, dom_phase;      // [nd]
  std::vector<uint8_t> reg_dom;                     // [nr] when nd > 0
  uint32_t n_signals() const { return ni + nr + nc + no; }
  uint32_t op_base() const { return ni + nr + nc; }
};

// Returns true on success; on failure err describes the first violation.
bool parse_netlist(const void* bytes, size_t nbytes, Netlist& out, std::string& err);

struct OpMeta {  // 16 bytes, one per lowered op (device uint4)
  uint32_t a, b, c, ctl;
};

struct Lowered {
  uint32_t n_slots = 0;
  // compact layout: rows of each width class in their own region (u64, u32,
  // u16, u8 in that order); inside a region, pool rows in signal order, then
  // op rows in slot order
  std::vector<uint32_t> slot_ref;        // [n_slots] row reference of every slot
  std::vector<uint32_t> dst_ref;         // [n_lowered] row reference of each op's output
  std::vector<uint32_t> reg_ref;         // [n_regs] row reference of Q
  std::vector<uint32_t> in_ref;          // [n_inputs]
  std::vector<uint32_t> const_ref;       // [n_consts]
  uint64_t lane_bytes = 0;               // bytes of state per lane
  uint32_t class_rows[4] = {0, 0, 0, 0};
  uint32_t input_base = 0, reg_base = 0, const_base = 0, op_base = 0;  // slot bases
  std::vector<uint32_t> sig2slot;        // [n_signals]
  std::vector<OpMeta> meta;              // [n_lowered] in slot order
  std::vector<uint32_t> ext_args;        // operand row references of ops with > 3 operands
  std::vector<uint32_t> layer_off;       // [n_layers + 1] into meta
  std::vector<uint32_t> layer_ext;       // [n_layers] first op of the layer with > 3 operands
                                         //   (they close the layer), or the layer's end
  std::vector<uint32_t> layer_wide;      // [n_layers] first op of the layer with <= 3 operands
                                         //   that is not narrow (narrow ones come first), or layer_ext
  std::vector<uint32_t> group_off;       // [n_groups + 1] into meta ((layer, opcode, width) runs)
  std::vector<uint32_t> reg_src;         // [n_regs] row reference of D (always an op row)
  std::vector<uint32_t> reg_width;       // [n_regs]
  std::vector<uint64_t> reg_init;        // [n_regs]
  std::vector<uint32_t> in_width;        // [n_inputs]
  std::vector<uint64_t> const_value;     // [n_consts] masked
  std::vector<uint32_t> mem_info;        // [n_mems][4] = word offset, words-1, width, first port
  std::vector<uint32_t> wport;           // [n_wports][4] = mem, en, addr, data (row references),
                                         //   sorted by memory, port order kept
  uint64_t mem_words_total = 0;
  uint64_t op_operands = 0;              // sum of operand counts over netlist ops
  uint32_t n_copies = 0;                 // copies inserted for edge sources
  uint32_t n_fused = 0;                  // muxes absorbed into mux chains
  uint32_t max_layer_ops = 0;
  // per-op-eval algorithmic bytes bookkeeping: sum over lowered ops of operands read
  uint64_t lowered_operands = 0;
};

// Multi-clock lowering (clock domains -> one clock): a hidden 32-bit register t
// (init 0, next t + 1) counts the non-reset cycles since reset; a register of a
// domain with period p > 1 and phase f loads through a hold mux enabled when
// ((t + f) & (p - 1)) == 0.  Returns the single-clock netlist; user2x maps the
// input's signal ids to its ids (the hidden signals come after them in each
// section).  Without domains (or all periods 1) the netlist is unchanged.
Netlist lower_clock_domains(const Netlist& nl, std::vector<uint32_t>& user2x);

// fuse_mux_chains: operator fusion of single-fanout mux chains into MUXCHAIN ops
// (the absorbed muxes are not computed and their signals have no row).
void lower_netlist(const Netlist& nl, Lowered& out, bool fuse_mux_chains = false);

// Design-specialised form (specialize.cpp): straight-line CUDA source of one
// thread simulating one lane for all cycles of a step, and its NVRTC compile
// for `arch` (e.g. "sm_103a").  compile returns false with the log on failure.
std::string specialized_source(const Netlist& nl, const Lowered& L);
// optimize: run the NVVM optimiser (its time grows superlinearly with the length).
bool compile_specialized(const std::string& src, const char* arch, bool optimize, std::vector<char>& cubin,
                         std::string& log);

}  // namespace rteaal
