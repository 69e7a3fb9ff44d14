// Host-only inspection of the lowering (no device, nothing kept): the entry
// points that expose what the kernels will execute -- the lowering's figures,
// the compact layout's row references, the one-clock netlist of the clock-domain
// lowering and the descriptors decoded back into a netlist -- so that all of it
// can be checked against the oracle without a GPU.  Also the FLOW form's tables
// (flow_tables, which the runtime uploads as they are built here) and the
// thread-local failure message of every entry point (rteaal_last_error).  Plain
// C++: this unit and lower.cpp build without the CUDA toolkit.
#include <algorithm>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "host_api.hpp"
#include "flow_tables.hpp"
#include "lower.hpp"

namespace rteaal {

void flow_tables(const Lowered& L, std::vector<uint32_t>& op, std::vector<uint32_t>& ext,
                 std::vector<uint32_t>& pool) {
  // region of each class in the compact layout (class 3 first) and the first
  // op row of each class (inside a class, pool rows come before op rows)
  const uint64_t c3 = L.class_rows[3], c2 = L.class_rows[2], c1 = L.class_rows[1];
  const uint64_t coff[4] = {8 * c3 + 4 * c2 + 2 * c1, 8 * c3 + 4 * c2, 8 * c3, 0};
  const uint64_t cidx[4] = {c3 + c2 + c1, c3 + c2, c3, 0};
  uint32_t op_off[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
  for (uint32_t sl = L.op_base; sl < L.n_slots; sl++) {
    const uint32_t k = L.slot_ref[sl] >> 30;
    op_off[k] = std::min(op_off[k], L.slot_ref[sl] & REF_OFF_MASK);
  }
  auto row_of = [&](uint32_t ref) {
    const uint32_t k = ref >> 30, off = ref & REF_OFF_MASK;
    return (uint32_t)(cidx[k] + ((off - coff[k]) >> k)) | (off >= op_off[k] ? FLOW_CHECK : 0u);
  };
  op.assign(8 * L.meta.size(), 0u);
  for (size_t i = 0; i < L.meta.size(); i++) {
    const OpMeta& m = L.meta[i];
    uint32_t* q = &op[8 * i];
    q[3] = row_of(L.dst_ref[i]) & ~FLOW_CHECK;
    q[4] = m.ctl;
    q[5] = L.dst_ref[i];
    if (m.ctl & CTL_EXT) {
      q[6] = m.a;
      q[7] = m.b;
    } else {
      const uint32_t ar = (m.ctl >> 5) & 3u;
      q[0] = row_of(m.a);
      q[1] = ar >= 2 ? row_of(m.b) : 0u;
      q[2] = ar >= 3 ? row_of(m.c) : 0u;
    }
  }
  ext.resize(L.ext_args.size());
  for (size_t k = 0; k < L.ext_args.size(); k++) ext[k] = row_of(L.ext_args[k]);
  pool.clear();
  for (const std::vector<uint32_t>* v : {&L.in_ref, &L.reg_ref, &L.const_ref})
    for (uint32_t r : *v) {
      pool.push_back(r);
      pool.push_back(row_of(r) & ~FLOW_CHECK);
    }
}


std::string& last_error() {
  thread_local std::string msg;
  return msg;
}

void fill_stats(const Netlist& nl, const Lowered& L, uint64_t metadata_bytes, rteaal_design_stats* o) {
  o->n_signals = nl.n_signals();
  o->n_inputs = nl.ni;
  o->n_regs = nl.nr;
  o->n_consts = nl.nc;
  o->n_ops = nl.no;
  o->n_mems = nl.nm;
  o->n_wports = nl.nw;
  o->n_layers = (uint32_t)L.layer_off.size() - 1;
  o->n_groups = (uint32_t)L.group_off.size() - 1;
  o->n_slots = L.n_slots;
  o->n_lowered_ops = (uint32_t)L.meta.size();
  o->max_layer_ops = L.max_layer_ops;
  o->op_operands = L.op_operands;
  o->mem_words_total = L.mem_words_total;
  o->metadata_bytes = metadata_bytes;
  o->state_bytes_per_lane = L.lane_bytes;
  o->n_fused = L.n_fused;
}

}  // namespace rteaal

using namespace rteaal;

RT_EXPORT const char* rteaal_last_error(void) { return last_error().c_str(); }

namespace {

// RTLN bytes of a netlist (the inverse of parse_netlist; layout in rteaal.h).
std::vector<uint8_t> serialize_netlist(const Netlist& nl) {
  std::vector<uint8_t> out;
  auto put = [&](const void* p, size_t n) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    out.insert(out.end(), b, b + n);
  };
  auto vec = [&](const auto& v) { put(v.data(), v.size() * sizeof(v[0])); };
  const uint32_t hdr[10] = {0x4E4C5452u, 1u, nl.ni, nl.nr, nl.nc, nl.no, nl.nm, nl.nw, nl.na, nl.nd};
  put(hdr, sizeof(hdr));
  vec(nl.reg_init);
  vec(nl.const_value);
  vec(nl.reg_d);
  vec(nl.argoff);
  vec(nl.args);
  vec(nl.mem_words);
  vec(nl.wport);
  if (nl.nd) {
    vec(nl.dom_period);
    vec(nl.dom_phase);
  }
  vec(nl.in_w);
  vec(nl.reg_w);
  vec(nl.const_w);
  vec(nl.code);
  vec(nl.width);
  vec(nl.p0);
  vec(nl.p1);
  vec(nl.mem_w);
  if (nl.nd) vec(nl.reg_dom);
  return out;
}

// The lowered design as a netlist: one signal per state row (the pool rows keep
// their ids, op rows follow in lowered order), every op decoded back from its
// descriptor (ctl word and operand row references, or its side-array operand
// list), registers and write ports from the clock-edge tables.
Netlist netlist_of_lowering(const Netlist& nlx, const Lowered& L) {
  std::unordered_map<uint32_t, uint32_t> slot_of_ref;
  for (uint32_t sl = 0; sl < L.n_slots; sl++) slot_of_ref[L.slot_ref[sl]] = sl;
  auto slot = [&](uint32_t ref) {
    auto it = slot_of_ref.find(ref);
    if (it == slot_of_ref.end()) throw Error(RTEAAL_E_FORMAT, "lowering: operand row without a slot");
    return it->second;
  };
  Netlist x;
  x.ni = nlx.ni;
  x.nc = nlx.nc;
  x.nr = (uint32_t)L.reg_src.size();
  x.in_w = nlx.in_w;
  x.const_w = nlx.const_w;
  x.const_value = L.const_value;
  for (uint32_t r = 0; r < x.nr; r++) {
    x.reg_w.push_back((uint8_t)L.reg_width[r]);
    x.reg_init.push_back(L.reg_init[r]);
    x.reg_d.push_back(slot(L.reg_src[r]));
  }
  x.argoff.push_back(0);
  for (const OpMeta& m : L.meta) {
    const uint32_t ctl = m.ctl;
    x.code.push_back((uint8_t)(ctl & 31u));
    x.width.push_back((uint8_t)((ctl >> 8) & 127u));
    x.p0.push_back((uint8_t)((ctl >> 16) & 255u));
    x.p1.push_back((uint8_t)(ctl >> 24));
    if (ctl & CTL_EXT) {
      for (uint32_t j = 0; j < m.b; j++) x.args.push_back(slot(L.ext_args[m.a + j]));
    } else {
      const uint32_t refs[3] = {m.a, m.b, m.c}, ar = (ctl >> 5) & 3u;
      for (uint32_t j = 0; j < ar; j++) x.args.push_back(slot(refs[j]));
    }
    x.argoff.push_back((uint32_t)x.args.size());
  }
  x.no = (uint32_t)L.meta.size();
  x.na = (uint32_t)x.args.size();
  x.nm = (uint32_t)(L.mem_info.size() / 4 - 1);
  for (uint32_t m = 0; m < x.nm; m++) {
    x.mem_words.push_back(L.mem_info[4ull * m + 1] + 1u);
    x.mem_w.push_back((uint8_t)L.mem_info[4ull * m + 2]);
  }
  x.nw = (uint32_t)(L.wport.size() / 4);
  for (uint32_t q = 0; q < x.nw; q++) {
    x.wport.push_back(L.wport[4ull * q]);
    for (int t = 1; t < 4; t++) x.wport.push_back(slot(L.wport[4ull * q + t]));
  }
  return x;
}

}  // namespace

RT_EXPORT int rteaal_design_lowered_netlist(const void* netlist, size_t nbytes, const rteaal_load_opts* opts,
                                            void* out, size_t capacity, size_t* out_bytes, uint32_t* user2sig,
                                            uint64_t n_user) {
  return guarded([&] {
    require(netlist && out_bytes, "rteaal_design_lowered_netlist: null argument");
    Netlist nl;
    std::string err;
    if (!parse_netlist(netlist, nbytes, nl, err)) throw Error(RTEAAL_E_FORMAT, err);
    std::vector<uint32_t> user2x;
    const Netlist nlx = lower_clock_domains(nl, user2x);
    Lowered L;
    lower_netlist(nlx, L, opts && opts->fuse_mux_chains);
    const std::vector<uint8_t> bytes = serialize_netlist(netlist_of_lowering(nlx, L));
    *out_bytes = bytes.size();
    if (out) {
      require(capacity >= bytes.size(), "rteaal_design_lowered_netlist: output buffer too small");
      std::memcpy(out, bytes.data(), bytes.size());
    }
    if (user2sig) {
      require(n_user == user2x.size(), "rteaal_design_lowered_netlist: n_user differs from the netlist's signal count");
      for (size_t i = 0; i < user2x.size(); i++) user2sig[i] = L.sig2slot[user2x[i]];
    }
  });
}

RT_EXPORT int rteaal_design_rows(const void* netlist, size_t nbytes, const rteaal_load_opts* opts, uint32_t* refs,
                                 uint64_t n_rows) {
  return guarded([&] {
    require(netlist && refs, "rteaal_design_rows: null argument");
    Netlist nl;
    std::string err;
    if (!parse_netlist(netlist, nbytes, nl, err)) throw Error(RTEAAL_E_FORMAT, err);
    std::vector<uint32_t> user2x;
    const Netlist nlx = lower_clock_domains(nl, user2x);
    Lowered L;
    lower_netlist(nlx, L, opts && opts->fuse_mux_chains);
    require(n_rows == L.n_slots, "rteaal_design_rows: n_rows differs from the lowered design's row count");
    std::copy(L.slot_ref.begin(), L.slot_ref.end(), refs);
  });
}

RT_EXPORT int rteaal_design_flow_tables(const void* netlist, size_t nbytes, const rteaal_load_opts* opts,
                                        uint32_t* op, uint64_t* n_op, uint32_t* ext, uint64_t* n_ext, uint32_t* pool,
                                        uint64_t* n_pool) {
  return guarded([&] {
    require(netlist && n_op && n_ext && n_pool, "rteaal_design_flow_tables: null argument");
    Netlist nl;
    std::string err;
    if (!parse_netlist(netlist, nbytes, nl, err)) throw Error(RTEAAL_E_FORMAT, err);
    std::vector<uint32_t> user2x;
    const Netlist nlx = lower_clock_domains(nl, user2x);
    Lowered L;
    lower_netlist(nlx, L, opts && opts->fuse_mux_chains);
    std::vector<uint32_t> o, e, p;
    flow_tables(L, o, e, p);
    if (op) {
      require(*n_op == o.size() / 8, "rteaal_design_flow_tables: n_op differs from the lowered op count");
      std::copy(o.begin(), o.end(), op);
    }
    if (ext) {
      require(*n_ext == e.size(), "rteaal_design_flow_tables: n_ext differs from the side array's length");
      std::copy(e.begin(), e.end(), ext);
    }
    if (pool) {
      require(*n_pool == p.size() / 2, "rteaal_design_flow_tables: n_pool differs from the pool row count");
      std::copy(p.begin(), p.end(), pool);
    }
    *n_op = o.size() / 8;
    *n_ext = e.size();
    *n_pool = p.size() / 2;
  });
}

RT_EXPORT int rteaal_design_single_clock(const void* netlist, size_t nbytes, void* out, size_t capacity,
                                         size_t* out_bytes, uint32_t* user2x, uint64_t n_user) {
  return guarded([&] {
    require(netlist && out_bytes, "rteaal_design_single_clock: null argument");
    Netlist nl;
    std::string err;
    if (!parse_netlist(netlist, nbytes, nl, err)) throw Error(RTEAAL_E_FORMAT, err);
    std::vector<uint32_t> map;
    const std::vector<uint8_t> bytes = serialize_netlist(lower_clock_domains(nl, map));
    *out_bytes = bytes.size();
    if (out) {
      require(capacity >= bytes.size(), "rteaal_design_single_clock: output buffer too small");
      std::memcpy(out, bytes.data(), bytes.size());
    }
    if (user2x) {
      require(n_user == map.size(), "rteaal_design_single_clock: n_user differs from the netlist's signal count");
      std::copy(map.begin(), map.end(), user2x);
    }
  });
}

RT_EXPORT int rteaal_design_lower(const void* netlist, size_t nbytes, const rteaal_load_opts* opts,
                                  rteaal_design_stats* o, uint32_t* layer_ops, uint32_t max_layers) {
  return guarded([&] {
    require(netlist && o, "rteaal_design_lower: null argument");
    Netlist nl;
    std::string err;
    if (!parse_netlist(netlist, nbytes, nl, err)) throw Error(RTEAAL_E_FORMAT, err);
    std::vector<uint32_t> user2x;
    const Netlist nlx = lower_clock_domains(nl, user2x);
    Lowered L;
    lower_netlist(nlx, L, opts && opts->fuse_mux_chains);
    fill_stats(nl, L, 0, o);
    if (layer_ops)
      for (uint32_t l = 0; l + 1 < L.layer_off.size() && l < max_layers; l++)
        layer_ops[l] = L.layer_off[l + 1] - L.layer_off[l];
  });
}

