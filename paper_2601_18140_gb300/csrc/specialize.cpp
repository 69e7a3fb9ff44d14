// specialize.cpp -- the design-specialised form: the paper's S-rank unrolling
// and tensor inlining (Sec. 5.2, kernels SU and TI) carried to the GPU.
//
// The lowered operation list is unrolled into straight-line CUDA source in
// which every signal is a local variable (the OIM is encoded in the code, no
// descriptors are read) and compiled at run time with NVRTC for sm_103a.  One
// thread simulates one instance (lane) for all the cycles of a step, so no
// barrier is needed between layers: the cascade's layer order is the
// topological order of the statements.  State rows are read once at the start
// of a step (inputs, registers) and every signal's row is written once at the
// end (the last cycle's values), in the same compact layout the data-driven
// kernels use, so forms can be switched between steps.  Semantics are those of
// include/rteaal.h; every result is masked to its width.
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <sstream>
#include <stdexcept>
#include <string>
#include <vector>

#include "lower.hpp"

namespace rteaal {

namespace {

std::string hex(uint64_t v) {
  char b[32];
  std::snprintf(b, sizeof b, "0x%llxull", (unsigned long long)v);
  return b;
}

uint64_t mask_of(uint32_t w) { return w >= 64 ? ~0ull : (1ull << w) - 1ull; }

struct Gen {
  const Netlist& nl;
  const Lowered& L;
  std::vector<uint8_t> sw;  // signal widths
  std::ostringstream o;

  explicit Gen(const Netlist& n, const Lowered& l) : nl(n), L(l) {
    sw.resize(nl.n_signals());
    for (uint32_t i = 0; i < nl.ni; i++) sw[i] = nl.in_w[i];
    for (uint32_t i = 0; i < nl.nr; i++) sw[nl.ni + i] = nl.reg_w[i];
    for (uint32_t i = 0; i < nl.nc; i++) sw[nl.ni + nl.nr + i] = nl.const_w[i];
    for (uint32_t k = 0; k < nl.no; k++) sw[nl.op_base() + k] = nl.width[k];
  }

  const char* ty(uint32_t sig) const { return sw[sig] <= 32 ? "u32" : "u64"; }
  std::string v(uint32_t sig) const { return "s" + std::to_string(sig); }
  std::string w(uint32_t sig) const { return "((u64)s" + std::to_string(sig) + ")"; }  // widened operand

  // expression of netlist op k (64-bit, before the width mask)
  std::string expr(uint32_t k) const {
    const uint32_t* a = &nl.args[nl.argoff[k]];
    const uint32_t n = nl.argoff[k + 1] - nl.argoff[k];
    const uint32_t p0 = nl.p0[k], p1 = nl.p1[k];
    auto fold = [&](const char* opr) {
      std::string e = w(a[0]);
      for (uint32_t i = 1; i < n; i++) e = "(" + e + " " + opr + " " + w(a[i]) + ")";
      return e;
    };
    switch (nl.code[k]) {
      case OP_COPY: return w(a[0]);
      case OP_AND: return fold("&");
      case OP_OR: return fold("|");
      case OP_XOR: return fold("^");
      case OP_NOT: return "(~" + w(a[0]) + ")";
      case OP_ADD: return fold("+");
      case OP_SUB: return "(" + w(a[0]) + " - " + w(a[1]) + ")";
      case OP_MUL: return fold("*");
      case OP_SHL: return p0 >= 64 ? std::string("0ull") : "(" + w(a[0]) + " << " + std::to_string(p0) + ")";
      case OP_SHR: return p0 >= 64 ? std::string("0ull") : "(" + w(a[0]) + " >> " + std::to_string(p0) + ")";
      case OP_DSHL: return "(" + w(a[1]) + " >= 64ull ? 0ull : " + w(a[0]) + " << (u32)" + w(a[1]) + ")";
      case OP_DSHR: return "(" + w(a[1]) + " >= 64ull ? 0ull : " + w(a[0]) + " >> (u32)" + w(a[1]) + ")";
      case OP_BITS: return "((" + w(a[0]) + " >> " + std::to_string(p1) + ") & " + hex(mask_of(p0 - p1 + 1)) + ")";
      case OP_CAT:
        return p0 >= 64 ? w(a[1]) : "((" + w(a[0]) + " << " + std::to_string(p0) + ") | " + w(a[1]) + ")";
      case OP_EQ: return "(u64)(" + w(a[0]) + " == " + w(a[1]) + ")";
      case OP_NEQ: return "(u64)(" + w(a[0]) + " != " + w(a[1]) + ")";
      case OP_LT: return "(u64)(" + w(a[0]) + " < " + w(a[1]) + ")";
      case OP_LEQ: return "(u64)(" + w(a[0]) + " <= " + w(a[1]) + ")";
      case OP_GT: return "(u64)(" + w(a[0]) + " > " + w(a[1]) + ")";
      case OP_GEQ: return "(u64)(" + w(a[0]) + " >= " + w(a[1]) + ")";
      case OP_MUX: return "((" + w(a[0]) + " & 1ull) ? " + w(a[1]) + " : " + w(a[2]) + ")";
      case OP_ANDR: return "(u64)((" + w(a[0]) + " & " + hex(mask_of(p0)) + ") == " + hex(mask_of(p0)) + ")";
      case OP_ORR: return "(u64)(" + w(a[0]) + " != 0ull)";
      case OP_XORR: return "(u64)(__popcll(" + w(a[0]) + ") & 1)";
      case OP_MEMRD: {
        const uint32_t mi = p0 | (p1 << 8);
        const uint32_t off = L.mem_info[4ull * mi], wm = L.mem_info[4ull * mi + 1];
        return "mem[((usz)" + std::to_string(off) + "u + (" + w(a[0]) + " & " + hex(wm) + ")) * np + lane]";
      }
      case OP_MUXCHAIN: {  // s0, v0, s1, v1, ..., default: the first set selector wins
        std::string e = w(a[n - 1]);
        for (int i = (int)n - 3; i >= 0; i -= 2) e = "((" + w(a[i]) + " & 1ull) ? " + w(a[i + 1]) + " : " + e + ")";
        return e;
      }
      default: throw std::runtime_error("specialize: unknown opcode");
    }
  }

  // load / store of a row (row reference) at this lane
  std::string ld(uint32_t ref) const {
    const uint32_t k = ref >> 30, off = ref & REF_OFF_MASK;
    static const char* T[4] = {"u8", "u16", "u32", "u64"};
    return std::string("(*(const ") + T[k] + "*)(st + (usz)" + std::to_string(off) + "u * np + ((usz)lane << " +
           std::to_string(k) + ")))";
  }
  std::string st(uint32_t ref, const std::string& val) const {
    const uint32_t k = ref >> 30, off = ref & REF_OFF_MASK;
    static const char* T[4] = {"u8", "u16", "u32", "u64"};
    return std::string("*(") + T[k] + "*)(st + (usz)" + std::to_string(off) + "u * np + ((usz)lane << " +
           std::to_string(k) + ")) = (" + T[k] + ")(" + val + ");";
  }
  uint32_t ref_of(uint32_t sig) const {
    const uint32_t slot = L.sig2slot[sig];
    return slot == 0xFFFFFFFFu ? 0xFFFFFFFFu : L.slot_ref[slot];
  }

  // one cycle: stimulus, every op in topological order, then the clock edge;
  // with store_ops, each op's value is also written to its row (last cycle)
  void cycle(bool store_ops) {
    const uint32_t opb = nl.op_base();
    o << "    if (stim_mode == 1) {\n";
    for (uint32_t i = 0; i < nl.ni; i++)
      o << "      x" << i << " ^= x" << i << " << 13; x" << i << " ^= x" << i << " >> 7; x" << i << " ^= x" << i
        << " << 17; " << v(i) << " = (" << ty(i) << ")(x" << i << " & " << hex(mask_of(nl.in_w[i])) << ");\n";
    o << "    } else if (stim_mode == 2) {\n";
    for (uint32_t i = 0; i < nl.ni; i++)
      o << "      " << v(i) << " = (" << ty(i) << ")(stim[((usz)c * " << nl.ni << "u + " << i
        << "u) * n_user + user] & " << hex(mask_of(nl.in_w[i])) << ");\n";
    o << "    }\n";
    for (uint32_t k = 0; k < nl.no; k++) {
      const uint32_t sig = opb + k;
      o << "    " << v(sig) << " = (" << ty(sig) << ")(" << expr(k) << " & " << hex(mask_of(nl.width[k])) << ");\n";
      if (store_ops) {
        const uint32_t r = ref_of(sig);
        if (r != 0xFFFFFFFFu) o << "    " << st(r, v(sig)) << "\n";
      }
    }
    o << "    {\n      const bool rs = reset || c < rl;\n";
    // memory write ports: pre-edge values, in port order
    for (uint32_t q = 0; q < nl.nw; q++) {
      const uint32_t m = nl.wport[4ull * q], en = nl.wport[4ull * q + 1], ad = nl.wport[4ull * q + 2],
                     da = nl.wport[4ull * q + 3];
      const uint32_t off = L.mem_info[4ull * m], wm = L.mem_info[4ull * m + 1], mw = L.mem_info[4ull * m + 2];
      o << "      if (" << w(en) << " & 1ull) mem[((usz)" << off << "u + (" << w(ad) << " & " << hex(wm)
        << ")) * np + lane] = " << w(da) << " & " << hex(mask_of(mw)) << ";\n";
    }
    for (uint32_t r = 0; r < nl.nr; r++) {
      const uint32_t q = nl.ni + r;
      o << "      const " << ty(q) << " n" << r << " = rs ? (" << ty(q) << ")" << hex(nl.reg_init[r] & mask_of(nl.reg_w[r]))
        << " : (" << ty(q) << ")(" << w(nl.reg_d[r]) << " & " << hex(mask_of(nl.reg_w[r])) << ");\n";
    }
    for (uint32_t r = 0; r < nl.nr; r++) o << "      " << v(nl.ni + r) << " = n" << r << ";\n";
    o << "    }\n";
  }

  std::string source() {
    const uint32_t opb = nl.op_base();
    o << "// generated: design-specialised cycle kernel (" << nl.no << " ops, " << nl.nr << " registers)\n"
      << "typedef unsigned long long u64; typedef unsigned int u32; typedef unsigned short u16;"
         " typedef unsigned char u8;\n"
      << "typedef unsigned long long usz;\n"
      << "extern \"C\" __global__ void __launch_bounds__(128) rteaal_spec(\n"
      << "    u8* __restrict__ st, u64* __restrict__ mem, u64* __restrict__ xs, const u64* __restrict__ stim,\n"
      << "    const u32* __restrict__ budget, const u32* __restrict__ reset_lane,\n"
      << "    const u32* __restrict__ user_of_lane, u32 np, u32 n_user, u32 uniform, int stim_mode, int reset) {\n"
      << "  const u32 lane = blockIdx.x * blockDim.x + threadIdx.x;\n"
      << "  if (lane >= np) return;\n"
      << "  const u32 ncyc = budget ? budget[lane] : (lane < n_user ? uniform : 0u);\n"
      << "  if (ncyc == 0u) return;\n"
      << "  const u32 rl = reset_lane ? reset_lane[lane] : 0u;\n"
      << "  const u32 user = user_of_lane ? user_of_lane[lane] : lane;\n"
      << "  (void)user; (void)stim; (void)mem; (void)rl;\n";
    for (uint32_t i = 0; i < nl.ni; i++) {
      o << "  " << ty(i) << " " << v(i) << " = " << ld(ref_of(i)) << ";\n";
      o << "  u64 x" << i << " = stim_mode == 1 ? xs[(usz)" << i << "u * np + lane] : 0ull;\n";
    }
    for (uint32_t r = 0; r < nl.nr; r++) o << "  " << ty(nl.ni + r) << " " << v(nl.ni + r) << " = " << ld(ref_of(nl.ni + r)) << ";\n";
    for (uint32_t c = 0; c < nl.nc; c++) {
      const uint32_t sig = nl.ni + nl.nr + c;
      o << "  const " << ty(sig) << " " << v(sig) << " = (" << ty(sig) << ")" << hex(nl.const_value[c] & mask_of(nl.const_w[c]))
        << ";\n";
    }
    for (uint32_t k = 0; k < nl.no; k++) o << "  " << ty(opb + k) << " " << v(opb + k) << ";\n";
    o << "  for (u32 c = 0; c + 1u < ncyc; c++) {\n";
    cycle(false);
    o << "  }\n  {\n    const u32 c = ncyc - 1u;\n";
    cycle(true);
    o << "  }\n";
    for (uint32_t i = 0; i < nl.ni; i++) {
      o << "  " << st(ref_of(i), v(i)) << "\n";
      o << "  if (stim_mode == 1) xs[(usz)" << i << "u * np + lane] = x" << i << ";\n";
    }
    for (uint32_t r = 0; r < nl.nr; r++) o << "  " << st(ref_of(nl.ni + r), v(nl.ni + r)) << "\n";
    o << "}\n";
    return o.str();
  }
};

}  // namespace

std::string specialized_source(const Netlist& nl, const Lowered& L) { return Gen(nl, L).source(); }

bool compile_specialized(const std::string& src, const char* arch, bool optimize, std::vector<char>& cubin,
                         std::string& log) {
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "rteaal_spec.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    log = "nvrtcCreateProgram failed";
    return false;
  }
  const std::string a = std::string("--gpu-architecture=") + arch;
  // Every signal is a local: ptxas gives the body 255 registers (8 warps per
  // SM), and capping them (launch bounds with 4 or 8 CTAs per SM) measured
  // slower -- the straight-line code has enough independent work per warp.
  // The NVVM optimiser cuts the instructions by 40 % (1.4x faster on a 2k-op
  // design) but its time grows superlinearly with the body, so long designs
  // go without it (ptxas still optimises).  RTEAAL_SPEC_NVRTC_OPT adds one
  // more option.
  const char* extra = std::getenv("RTEAAL_SPEC_NVRTC_OPT");
  std::vector<const char*> opts = {a.c_str(), "--std=c++17", "-w"};
  if (!optimize) opts.push_back("-Xnvvm=-opt=0");
  if (extra) opts.push_back(extra);
  const nvrtcResult r = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
  size_t n = 0;
  nvrtcGetProgramLogSize(prog, &n);
  log.assign(n, '\0');
  if (n) nvrtcGetProgramLog(prog, &log[0]);
  bool ok = r == NVRTC_SUCCESS;
  if (ok) {
    size_t nb = 0;
    ok = nvrtcGetCUBINSize(prog, &nb) == NVRTC_SUCCESS && nb > 0;
    if (ok) {
      cubin.resize(nb);
      ok = nvrtcGetCUBIN(prog, cubin.data()) == NVRTC_SUCCESS;
    }
  }
  nvrtcDestroyProgram(&prog);
  return ok;
}

}  // namespace rteaal
