// lower.cpp -- RTLN parsing / validation and the lowering to device tensors.
#include "lower.hpp"

#include <algorithm>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <unordered_map>

namespace rteaal {

namespace {

template <typename T>
void take(const uint8_t*& p, std::vector<T>& v, size_t n) {
  v.resize(n);
  if (n) std::memcpy(v.data(), p, n * sizeof(T));
  p += n * sizeof(T);
}

bool fail(std::string& err, const std::string& msg) {
  err = msg;
  return false;
}

}  // namespace

bool parse_netlist(const void* bytes, size_t nbytes, Netlist& n, std::string& err) {
  if (!bytes || nbytes < 40) return fail(err, "netlist: shorter than the 40-byte header");
  uint32_t h[10];
  std::memcpy(h, bytes, sizeof(h));
  if (h[0] != 0x4E4C5452u) return fail(err, "netlist: bad magic (expected RTLN)");
  if (h[1] != 1u) return fail(err, "netlist: unsupported version");
  n.ni = h[2]; n.nr = h[3]; n.nc = h[4]; n.no = h[5]; n.nm = h[6]; n.nw = h[7]; n.na = h[8];
  n.nd = h[9];
  if (n.nd > 256) return fail(err, "netlist: more than 256 clock domains");
  const uint64_t need = 40ull + 8ull * n.nr + 8ull * n.nc + 4ull * n.nr + 4ull * (n.no + 1ull) +
                        4ull * n.na + 4ull * n.nm + 16ull * n.nw + 8ull * n.nd + n.ni + n.nr + n.nc +
                        4ull * n.no + n.nm + (n.nd ? n.nr : 0ull);
  if (need != nbytes) return fail(err, "netlist: size does not match the header counts");
  if ((uint64_t)n.ni + n.nr + n.nc + n.no >= 0x7FFFFFFFull)
    return fail(err, "netlist: too many signals");
  const uint8_t* p = static_cast<const uint8_t*>(bytes) + 40;
  take(p, n.reg_init, n.nr);
  take(p, n.const_value, n.nc);
  take(p, n.reg_d, n.nr);
  take(p, n.argoff, n.no + 1ull);
  take(p, n.args, n.na);
  take(p, n.mem_words, n.nm);
  take(p, n.wport, 4ull * n.nw);
  take(p, n.dom_period, n.nd);
  take(p, n.dom_phase, n.nd);
  take(p, n.in_w, n.ni);
  take(p, n.reg_w, n.nr);
  take(p, n.const_w, n.nc);
  take(p, n.code, n.no);
  take(p, n.width, n.no);
  take(p, n.p0, n.no);
  take(p, n.p1, n.no);
  take(p, n.mem_w, n.nm);
  take(p, n.reg_dom, n.nd ? n.nr : 0u);

  const uint32_t nsig = n.n_signals(), opb = n.op_base();
  auto wok = [](uint32_t w) { return w >= 1 && w <= 64; };
  for (uint32_t i = 0; i < n.ni; i++)
    if (!wok(n.in_w[i])) return fail(err, "netlist: input width outside 1..64");
  for (uint32_t i = 0; i < n.nr; i++) {
    if (!wok(n.reg_w[i])) return fail(err, "netlist: register width outside 1..64");
    if (n.reg_d[i] >= nsig) return fail(err, "netlist: register D is not a signal");
  }
  for (uint32_t i = 0; i < n.nc; i++)
    if (!wok(n.const_w[i])) return fail(err, "netlist: constant width outside 1..64");
  if (n.argoff[0] != 0 || n.argoff[n.no] != n.na)
    return fail(err, "netlist: operand offsets do not span the operand array");
  for (uint32_t m = 0; m < n.nm; m++) {
    const uint32_t w = n.mem_words[m];
    if (w == 0 || (w & (w - 1)) != 0) return fail(err, "netlist: memory words not a power of two");
    if (!wok(n.mem_w[m])) return fail(err, "netlist: memory width outside 1..64");
  }
  for (uint32_t k = 0; k < n.no; k++) {
    const uint32_t c = n.code[k], a0 = n.argoff[k], a1 = n.argoff[k + 1];
    if (a1 < a0) return fail(err, "netlist: operand offsets decrease");
    if (!wok(n.width[k])) return fail(err, "netlist: op width outside 1..64");
    if (c >= OP_COUNT) return fail(err, "netlist: unknown opcode");
    const uint32_t cnt = a1 - a0;
    for (uint32_t j = a0; j < a1; j++)
      if (n.args[j] >= opb + k) return fail(err, "netlist: operand not earlier in topological order");
    bool ok = true;
    switch (c) {
      case OP_AND: case OP_OR: case OP_XOR: case OP_ADD: case OP_MUL: ok = cnt >= 2; break;
      case OP_SUB: case OP_DSHL: case OP_DSHR: case OP_EQ: case OP_NEQ: case OP_LT: case OP_LEQ:
      case OP_GT: case OP_GEQ: ok = cnt == 2; break;
      case OP_CAT: ok = cnt == 2 && n.p0[k] >= 1 && n.p0[k] <= 64; break;
      case OP_MUX: ok = cnt == 3; break;
      case OP_MUXCHAIN: ok = cnt >= 3 && (cnt & 1u); break;
      case OP_BITS: ok = cnt == 1 && n.p0[k] >= n.p1[k] && n.p0[k] <= 63; break;
      case OP_ANDR: ok = cnt == 1 && n.p0[k] >= 1 && n.p0[k] <= 64; break;
      case OP_MEMRD: ok = cnt == 1 && (uint32_t)(n.p0[k] | (n.p1[k] << 8)) < n.nm; break;
      default: ok = cnt == 1; break;
    }
    if (!ok) return fail(err, "netlist: op " + std::to_string(k) + " has bad operands/params");
  }
  for (uint32_t q = 0; q < n.nw; q++) {
    const uint32_t* w = &n.wport[4ull * q];
    if (w[0] >= n.nm || w[1] >= nsig || w[2] >= nsig || w[3] >= nsig)
      return fail(err, "netlist: write port references a bad memory or signal");
  }
  for (uint32_t d = 0; d < n.nd; d++) {
    const uint32_t per = n.dom_period[d];
    if (per == 0 || per > (1u << 31) || (per & (per - 1)) != 0 || n.dom_phase[d] >= per)
      return fail(err, "netlist: clock domain period not a power of two, or phase >= period");
  }
  for (uint32_t r = 0; n.nd && r < n.nr; r++)
    if (n.reg_dom[r] >= n.nd) return fail(err, "netlist: register clock domain out of range");
  return true;
}

Netlist lower_clock_domains(const Netlist& nl, std::vector<uint32_t>& user2x) {
  const uint32_t nsig = nl.n_signals();
  user2x.resize(nsig);
  std::vector<uint32_t> gated;  // domains with period > 1
  for (uint32_t d = 0; d < nl.nd; d++)
    if (nl.dom_period[d] > 1) gated.push_back(d);
  if (gated.empty()) {
    for (uint32_t i = 0; i < nsig; i++) user2x[i] = i;
    Netlist x = nl;
    x.nd = 0;
    x.dom_period.clear();
    x.dom_phase.clear();
    x.reg_dom.clear();
    return x;
  }
  Netlist x;
  x.ni = nl.ni;
  x.nr = nl.nr + 1;                                      // + t
  const uint32_t n_extra_c = 2 + 2 * (uint32_t)gated.size();  // 1, 0, then per domain phase, p - 1
  x.nc = nl.nc + n_extra_c;
  x.nm = nl.nm;
  x.nw = nl.nw;
  const uint32_t t_sig = nl.ni + nl.nr;
  const uint32_t cbase = x.ni + x.nr, obase = cbase + x.nc;
  for (uint32_t i = 0; i < nsig; i++) {
    if (i < nl.ni + nl.nr) user2x[i] = i;
    else if (i < nl.op_base()) user2x[i] = i + 1;
    else user2x[i] = obase + (i - nl.op_base());
  }
  auto X = [&](uint32_t s) { return user2x[s]; };
  // constants: the input's, then 1, 0, and per gated domain its phase and p - 1
  x.const_value = nl.const_value;
  x.const_w = nl.const_w;
  const uint32_t c_one = cbase + nl.nc, c_zero = c_one + 1;
  x.const_value.push_back(1);
  x.const_w.push_back(32);
  x.const_value.push_back(0);
  x.const_w.push_back(1);
  for (uint32_t d : gated) {
    x.const_value.push_back(nl.dom_phase[d]);
    x.const_w.push_back(32);
    x.const_value.push_back(nl.dom_period[d] - 1u);
    x.const_w.push_back(32);
  }
  // ops: the input's (operands renumbered), then t + 1, the enables, the hold muxes
  x.code = nl.code;
  x.width = nl.width;
  x.p0 = nl.p0;
  x.p1 = nl.p1;
  x.argoff = nl.argoff;
  x.args.resize(nl.args.size());
  for (size_t j = 0; j < nl.args.size(); j++) x.args[j] = X(nl.args[j]);
  auto put = [&](uint32_t code, uint32_t w, std::initializer_list<uint32_t> a) {
    x.code.push_back((uint8_t)code);
    x.width.push_back((uint8_t)w);
    x.p0.push_back(0);
    x.p1.push_back(0);
    for (uint32_t v : a) x.args.push_back(v);
    x.argoff.push_back((uint32_t)x.args.size());
    return obase + (uint32_t)x.code.size() - 1u;
  };
  const uint32_t t_next = put(OP_ADD, 32, {t_sig, c_one});
  std::vector<uint32_t> enable(nl.nd, 0xFFFFFFFFu);
  for (size_t g = 0; g < gated.size(); g++) {
    const uint32_t d = gated[g];
    const uint32_t c_ph = c_zero + 1 + 2 * (uint32_t)g, c_mask = c_ph + 1;
    const uint32_t sum = nl.dom_phase[d] ? put(OP_ADD, 32, {t_sig, c_ph}) : t_sig;
    const uint32_t low = put(OP_AND, 32, {sum, c_mask});
    enable[d] = put(OP_EQ, 1, {low, c_zero});
  }
  x.reg_init = nl.reg_init;
  x.reg_init.push_back(0);
  x.reg_w = nl.reg_w;
  x.reg_w.push_back(32);
  x.reg_d.resize(x.nr);
  for (uint32_t r = 0; r < nl.nr; r++) {
    const uint32_t d = nl.reg_dom[r];
    x.reg_d[r] = enable[d] == 0xFFFFFFFFu ? X(nl.reg_d[r])
                                           : put(OP_MUX, nl.reg_w[r], {enable[d], X(nl.reg_d[r]), nl.ni + r});
  }
  x.reg_d[nl.nr] = t_next;
  x.no = (uint32_t)x.code.size();
  x.na = (uint32_t)x.args.size();
  x.in_w = nl.in_w;
  x.mem_words = nl.mem_words;
  x.mem_w = nl.mem_w;
  x.wport = nl.wport;
  for (uint32_t q = 0; q < nl.nw; q++)
    for (int t = 1; t < 4; t++) x.wport[4ull * q + t] = X(nl.wport[4ull * q + t]);
  return x;
}

void lower_netlist(const Netlist& nl, Lowered& L, bool fuse_mux_chains) {
  const uint32_t nsig = nl.n_signals(), opb = nl.op_base();
  constexpr uint32_t NONE = 0xFFFFFFFFu;

  // 0. operator fusion (optional): a MUX whose false operand (O = 2) is another
  //    MUX read nowhere else, and at least as wide, absorbs it; the chain becomes
  //    one MUXCHAIN s0, v0, s1, v1, ..., default.  Every absorbed width >= the head
  //    width, so the inner masks vanish under the head's mask.
  std::vector<uint32_t> fanout(nsig, 0);
  for (uint32_t j = 0; j < nl.na; j++) fanout[nl.args[j]]++;
  for (uint32_t r = 0; r < nl.nr; r++) fanout[nl.reg_d[r]]++;
  for (uint32_t q = 0; q < nl.nw; q++)
    for (int t = 1; t < 4; t++) fanout[nl.wport[4ull * q + t]]++;
  std::vector<uint8_t> absorbed(nl.no, 0);
  std::vector<uint32_t> head_args_off, head_args;  // CSR of fused operand lists (signal ids)
  std::vector<uint32_t> head_of(nl.no, NONE);      // netlist op -> index into head_args_off
  if (fuse_mux_chains) {
    auto fusable = [&](uint32_t sig, uint32_t head_w) {
      if (sig < opb) return false;
      const uint32_t k = sig - opb;
      return nl.code[k] == OP_MUX && fanout[sig] == 1 && nl.width[k] >= head_w;
    };
    head_args_off.push_back(0);
    for (int64_t kk = (int64_t)nl.no - 1; kk >= 0; kk--) {  // heads are found from the top down
      const uint32_t k = (uint32_t)kk;
      if (absorbed[k] || nl.code[k] != OP_MUX) continue;
      const uint32_t w0 = nl.width[k];
      uint32_t cur = k;
      if (!fusable(nl.args[nl.argoff[cur] + 2], w0)) continue;
      std::vector<uint32_t> a;
      for (;;) {
        const uint32_t* x = &nl.args[nl.argoff[cur]];
        a.push_back(x[0]);
        a.push_back(x[1]);
        if (!fusable(x[2], w0)) {
          a.push_back(x[2]);
          break;
        }
        cur = x[2] - opb;
        absorbed[cur] = 1;
      }
      head_of[k] = (uint32_t)head_args_off.size() - 1;
      head_args.insert(head_args.end(), a.begin(), a.end());
      head_args_off.push_back((uint32_t)head_args.size());
    }
  }
  auto op_args = [&](uint32_t k, std::vector<uint32_t>& out) {
    out.clear();
    if (head_of[k] != NONE)
      out.assign(head_args.begin() + head_args_off[head_of[k]], head_args.begin() + head_args_off[head_of[k] + 1]);
    else
      out.assign(nl.args.begin() + nl.argoff[k], nl.args.begin() + nl.argoff[k + 1]);
  };

  // 1. levelisation: level(pool) = 0, level(op) = 1 + max level of its operands.
  std::vector<uint32_t> level(nsig, 0);
  std::vector<uint32_t> tmp;
  for (uint32_t k = 0; k < nl.no; k++) {
    if (absorbed[k]) continue;
    op_args(k, tmp);
    uint32_t lv = 0;
    for (uint32_t x : tmp) lv = std::max(lv, level[x]);
    level[opb + k] = lv + 1;
  }

  // 2. lowered op list: netlist ops (fused heads as MUXCHAIN, absorbed muxes
  //    dropped) plus a COPY (level 1) for every register D or write-port signal
  //    that is not an op output, so that the clock edge reads only op slots (no
  //    hazard with the register writes or the next cycle's inputs).
  struct LOp {
    uint32_t level, code, width, p0, p1, src_sig;  // src_sig: netlist op index, or copy source
    bool is_copy;
    bool is_ext;  // more than three operands: operand rows in the side array
    bool wide;    // result or an operand wider than 32 bits, or MEMRD (see CTL_NARROW)
  };
  std::vector<LOp> ops;
  ops.reserve(nl.no + 16);
  std::vector<uint32_t> lop_of(nl.no, NONE);
  L.n_fused = 0;
  for (uint32_t k = 0; k < nl.no; k++) {
    if (absorbed[k]) {
      L.n_fused++;
      continue;
    }
    lop_of[k] = (uint32_t)ops.size();
    const uint32_t code = head_of[k] != NONE ? (uint32_t)OP_MUXCHAIN : nl.code[k];
    op_args(k, tmp);
    ops.push_back({level[opb + k], code, nl.width[k], nl.p0[k], nl.p1[k], k, false, tmp.size() > 3, false});
  }
  std::unordered_map<uint32_t, uint32_t> copy_of;  // pool signal -> lowered op index
  std::vector<uint8_t> sig_w(nsig);
  for (uint32_t i = 0; i < nl.ni; i++) sig_w[i] = nl.in_w[i];
  for (uint32_t i = 0; i < nl.nr; i++) sig_w[nl.ni + i] = nl.reg_w[i];
  for (uint32_t i = 0; i < nl.nc; i++) sig_w[nl.ni + nl.nr + i] = nl.const_w[i];
  for (uint32_t k = 0; k < nl.no; k++) sig_w[opb + k] = nl.width[k];
  auto edge_src = [&](uint32_t sig) -> int64_t {  // lowered op index that holds sig
    if (sig >= opb) return (int64_t)lop_of[sig - opb];
    auto it = copy_of.find(sig);
    if (it != copy_of.end()) return it->second;
    const uint32_t idx = (uint32_t)ops.size();
    ops.push_back({1u, OP_COPY, sig_w[sig], 0u, 0u, sig, true, false, false});
    copy_of[sig] = idx;
    return idx;
  };
  std::vector<int64_t> reg_lop(nl.nr);
  for (uint32_t r = 0; r < nl.nr; r++) reg_lop[r] = edge_src(nl.reg_d[r]);
  std::vector<int64_t> wp_lop(3ull * nl.nw);
  for (uint32_t q = 0; q < nl.nw; q++)
    for (int t = 0; t < 3; t++) wp_lop[3ull * q + t] = edge_src(nl.wport[4ull * q + 1 + t]);
  L.n_copies = (uint32_t)copy_of.size();
  // narrow ops (CTL_NARROW): the result and every operand fit 32 bits
  for (LOp& o : ops) {
    bool narrow = o.width <= 32 && o.code != OP_MEMRD && (o.code != OP_BITS || o.p0 < 32) &&
                  (o.code != OP_ANDR || o.p0 <= 32);
    if (o.is_copy) {
      narrow = narrow && sig_w[o.src_sig] <= 32;
    } else {
      op_args(o.src_sig, tmp);
      for (uint32_t x : tmp) narrow = narrow && sig_w[x] <= 32;
    }
    o.wide = !narrow;
  }

  // 3. order: by level, then ops with at most three operands before the others,
  //    and among those the narrow ones before the wide ones (so kernels walk
  //    each kind with its own loop), then (opcode, width) -- the N rank
  //    swizzled above S -- then original order.  Position = slot offset (S
  //    coordinates implicit).
  std::vector<uint32_t> order(ops.size());
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
    const LOp &a = ops[x], &b = ops[y];
    if (a.level != b.level) return a.level < b.level;
    if (a.is_ext != b.is_ext) return b.is_ext;
    if (!a.is_ext && a.wide != b.wide) return b.wide;
    if (a.code != b.code) return a.code < b.code;
    return a.width < b.width;
  });
  std::vector<uint32_t> pos(ops.size());
  for (uint32_t i = 0; i < order.size(); i++) pos[order[i]] = i;

  L.input_base = 0;
  L.reg_base = nl.ni;
  L.const_base = nl.ni + nl.nr;
  L.op_base = opb;
  L.n_slots = opb + (uint32_t)ops.size();
  L.sig2slot.resize(nsig);
  for (uint32_t s = 0; s < opb; s++) L.sig2slot[s] = s;
  for (uint32_t k = 0; k < nl.no; k++) L.sig2slot[opb + k] = lop_of[k] == NONE ? NONE : opb + pos[lop_of[k]];

  // 3b. compact layout: width class of every slot, row references
  {
    std::vector<uint32_t> cls(L.n_slots);
    for (uint32_t sgl = 0; sgl < opb; sgl++) cls[sgl] = width_class(sig_w[sgl]);
    for (uint32_t i = 0; i < order.size(); i++) cls[opb + i] = width_class(ops[order[i]].width);
    uint64_t cnt[4] = {0, 0, 0, 0};
    for (uint32_t sl = 0; sl < L.n_slots; sl++) cnt[cls[sl]]++;
    uint64_t base[4];
    base[3] = 0;
    base[2] = base[3] + 8 * cnt[3];
    base[1] = base[2] + 4 * cnt[2];
    base[0] = base[1] + 2 * cnt[1];
    L.lane_bytes = base[0] + cnt[0];
    if (L.lane_bytes > REF_OFF_MASK) throw std::runtime_error("design too large: > 1 GiB of state per instance");
    uint64_t next[4] = {base[0], base[1], base[2], base[3]};
    L.slot_ref.resize(L.n_slots);
    for (uint32_t sl = 0; sl < L.n_slots; sl++) {
      const uint32_t k = cls[sl];
      L.slot_ref[sl] = (k << 30) | (uint32_t)next[k];
      next[k] += 1ull << k;
    }
    for (int k = 0; k < 4; k++) L.class_rows[k] = (uint32_t)cnt[k];
  }
  auto ref_of_sig = [&](uint32_t sig) { return L.slot_ref[L.sig2slot[sig]]; };

  // 4. per-op metadata (operands as row references, ctl word)
  L.meta.resize(ops.size());
  L.ext_args.clear();
  L.lowered_operands = 0;
  L.op_operands = nl.na;
  uint32_t n_layers = 0;
  for (const LOp& o : ops) n_layers = std::max(n_layers, o.level);
  L.layer_off.assign(n_layers + 1, 0);
  L.layer_ext.assign(n_layers, NONE);
  L.layer_wide.assign(n_layers, NONE);
  L.group_off.clear();
  for (uint32_t i = 0; i < order.size(); i++) {
    const LOp& o = ops[order[i]];
    std::vector<uint32_t> a;
    uint32_t code = o.code;
    if (o.is_copy) {
      a.push_back(ref_of_sig(o.src_sig));
    } else {
      op_args(o.src_sig, tmp);
      for (uint32_t x : tmp) a.push_back(ref_of_sig(x));
      if (code == OP_MUXCHAIN && a.size() == 3) code = OP_MUX;  // one pair + default == mux
    }
    L.lowered_operands += a.size();
    OpMeta m{};
    uint32_t ctl = code | (o.width << 8) | (o.p0 << 16) | (o.p1 << 24);
    if (!o.wide) ctl |= CTL_NARROW;
    if (a.size() <= 3) {
      m.a = a[0];
      m.b = a.size() > 1 ? a[1] : a[0];
      m.c = a.size() > 2 ? a[2] : a[0];
      ctl |= (uint32_t)a.size() << 5;
    } else {
      m.a = (uint32_t)L.ext_args.size();
      m.b = (uint32_t)a.size();
      m.c = 0;
      L.ext_args.insert(L.ext_args.end(), a.begin(), a.end());
      ctl |= CTL_EXT;
    }
    m.ctl = ctl;
    L.meta[i] = m;
    if ((ctl & CTL_EXT) && L.layer_ext[o.level - 1] == NONE) L.layer_ext[o.level - 1] = i;
    if (!(ctl & CTL_EXT) && o.wide && L.layer_wide[o.level - 1] == NONE) L.layer_wide[o.level - 1] = i;
    L.layer_off[o.level] = i + 1;  // running end of the layer
    if (i == 0 || ops[order[i - 1]].level != o.level || ops[order[i - 1]].code != o.code ||
        ops[order[i - 1]].width != o.width)
      L.group_off.push_back(i);
  }
  L.group_off.push_back((uint32_t)order.size());
  L.dst_ref.resize(order.size());
  for (uint32_t i = 0; i < order.size(); i++) L.dst_ref[i] = L.slot_ref[opb + i];
  // layer_off[l] holds the end of level l (levels 1..n); shift to begin offsets
  std::vector<uint32_t> ends(L.layer_off.begin() + 1, L.layer_off.end());
  L.layer_off[0] = 0;
  for (uint32_t l = 0; l < n_layers; l++) L.layer_off[l + 1] = ends[l];
  for (uint32_t l = 0; l < n_layers; l++) {
    if (L.layer_ext[l] == NONE) L.layer_ext[l] = L.layer_off[l + 1];
    if (L.layer_wide[l] == NONE) L.layer_wide[l] = L.layer_ext[l];
  }
  L.max_layer_ops = 0;
  for (uint32_t l = 0; l < n_layers; l++)
    L.max_layer_ops = std::max(L.max_layer_ops, L.layer_off[l + 1] - L.layer_off[l]);

  // 5. clock-edge tables
  L.reg_src.resize(nl.nr);
  L.reg_width.resize(nl.nr);
  L.reg_init.resize(nl.nr);
  for (uint32_t r = 0; r < nl.nr; r++) {
    L.reg_src[r] = L.slot_ref[opb + pos[(uint32_t)reg_lop[r]]];
    L.reg_width[r] = nl.reg_w[r];
    L.reg_init[r] = nl.reg_init[r];
  }
  L.in_width.assign(nl.in_w.begin(), nl.in_w.end());
  L.reg_ref.resize(nl.nr);
  for (uint32_t r = 0; r < nl.nr; r++) L.reg_ref[r] = L.slot_ref[L.reg_base + r];
  L.in_ref.resize(nl.ni);
  for (uint32_t j = 0; j < nl.ni; j++) L.in_ref[j] = L.slot_ref[L.input_base + j];
  L.const_ref.resize(nl.nc);
  for (uint32_t c = 0; c < nl.nc; c++) L.const_ref[c] = L.slot_ref[L.const_base + c];
  L.const_value.resize(nl.nc);
  for (uint32_t c = 0; c < nl.nc; c++) {
    const uint32_t w = nl.const_w[c];
    L.const_value[c] = nl.const_value[c] & (~0ull >> (64 - w));
  }
  // memories and their write ports (grouped by memory, port order preserved)
  std::vector<uint32_t> pidx(nl.nw);
  std::iota(pidx.begin(), pidx.end(), 0u);
  std::stable_sort(pidx.begin(), pidx.end(),
                   [&](uint32_t x, uint32_t y) { return nl.wport[4ull * x] < nl.wport[4ull * y]; });
  L.wport.resize(4ull * nl.nw);
  for (uint32_t i = 0; i < nl.nw; i++) {
    const uint32_t q = pidx[i];
    L.wport[4ull * i + 0] = nl.wport[4ull * q];
    for (int t = 0; t < 3; t++) L.wport[4ull * i + 1 + t] = L.slot_ref[opb + pos[(uint32_t)wp_lop[3ull * q + t]]];
  }
  L.mem_info.assign(4ull * (nl.nm + 1), 0);
  uint64_t off = 0;
  uint32_t port = 0;
  for (uint32_t m = 0; m <= nl.nm; m++) {
    while (port < nl.nw && L.wport[4ull * port] < m) port++;
    L.mem_info[4ull * m + 0] = (uint32_t)off;
    L.mem_info[4ull * m + 1] = m < nl.nm ? nl.mem_words[m] - 1 : 0;
    L.mem_info[4ull * m + 2] = m < nl.nm ? nl.mem_w[m] : 0;
    L.mem_info[4ull * m + 3] = port;
    if (m < nl.nm) off += nl.mem_words[m];
  }
  L.mem_words_total = off;
}

}  // namespace rteaal
