/* oracle.c -- TEST INFRASTRUCTURE ONLY (never part of the product path).
 *
 * Plain, slow, gate-by-gate cycle-accurate RTL simulator used as the parity
 * oracle for the GPU path.  It implements the textbook definition of
 * full-cycle, activity-oblivious simulation of a synchronous single-clock
 * design (Sec. 2.1 and Fig. 1 of the paper: evaluate the dataflow graph, then
 * commit register next states at the clock edge), with no layers, no grouping
 * by operation type and no operation-input-mask tensors.  Each cycle, for each
 * instance:
 *   1. drive the primary inputs (the testbench writes the layer input at the
 *      cycle boundary, Sec. 6.2 "Host-DUT Communication");
 *   2. evaluate every operation in the netlist's topological order,
 *      v = f_op(v[operands], params) masked to the op's width;
 *   3. at the edge: every register takes reset ? init : v[D] (masked to its
 *      width); memory write ports apply in port order;
 *   4. the next cycle reads the new register values.
 * Clock domains (optional; the paper's multi-clock reading, Sec. 6.2 "Multiple
 * Clock Domains"): each instance counts t, the non-reset cycles completed since
 * its last reset cycle; at the edge of a non-reset cycle a register of domain
 * (period p, phase f) takes v[D] only if (t + f) mod p == 0, else it keeps its
 * value; a reset cycle resets every register and sets t = 0.
 * Operation semantics are the readings written down in include/rteaal.h
 * (UInt only, every value zero-extended in 64 bits, masked to its width).
 *
 * Shares no code with the CUDA library: it parses the RTLN netlist bytes
 * itself.  Instances are independent; threads split them.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  O_COPY = 0, O_AND, O_OR, O_XOR, O_NOT, O_ADD, O_SUB, O_MUL, O_SHL, O_SHR, O_DSHL, O_DSHR,
  O_BITS, O_CAT, O_EQ, O_NEQ, O_LT, O_LEQ, O_GT, O_GEQ, O_MUX, O_ANDR, O_ORR, O_XORR,
  O_MEMRD, O_MUXCHAIN, O_COUNT
};

typedef struct {
  uint32_t ni, nr, nc, no, nm, nw, na;
  uint32_t nsig, reg_base, const_base, op_base;
  uint64_t *buf; /* 8-byte aligned private copy of the netlist bytes */
  const uint64_t *reg_init, *const_value;
  const uint32_t *reg_d, *argoff, *args, *mem_words, *wport;
  const uint8_t *in_w, *reg_w, *const_w, *code, *width, *p0, *p1, *mem_w;
  uint32_t nd;                          /* clock domains (0: one clock)       */
  const uint32_t *dom_period, *dom_phase;
  const uint8_t *reg_dom;
  uint64_t *mem_off; /* word offset of each memory inside one instance's memory block */
  uint64_t mem_total;
} onl;

static uint64_t mask_w(unsigned w) { return w >= 64 ? ~0ull : ((1ull << w) - 1ull); }

static void onl_free(onl *n) {
  free(n->buf);
  free(n->mem_off);
  memset(n, 0, sizeof(*n));
}

/* Parse and validate.  Returns 0 or -2 (format error). */
static int onl_parse(const uint8_t *bytes, size_t nbytes, onl *n) {
  memset(n, 0, sizeof(*n));
  if (nbytes < 40) return -2;
  n->buf = (uint64_t *)malloc((nbytes + 7) & ~(size_t)7);
  if (!n->buf) return -2;
  memcpy(n->buf, bytes, nbytes);
  const uint32_t *h = (const uint32_t *)n->buf;
  if (h[0] != 0x4E4C5452u || h[1] != 1u) goto bad;
  n->ni = h[2]; n->nr = h[3]; n->nc = h[4]; n->no = h[5]; n->nm = h[6]; n->nw = h[7]; n->na = h[8];
  n->nd = h[9];
  {
    uint64_t need = 40 + 8ull * n->nr + 8ull * n->nc + 4ull * n->nr + 4ull * (n->no + 1ull) +
                    4ull * n->na + 4ull * n->nm + 16ull * n->nw + 8ull * n->nd + n->ni + n->nr +
                    n->nc + 4ull * n->no + n->nm + (n->nd ? n->nr : 0);
    if (need != nbytes) goto bad;
  }
  {
    const uint8_t *p = (const uint8_t *)n->buf + 40;
    n->reg_init = (const uint64_t *)p; p += 8ull * n->nr;
    n->const_value = (const uint64_t *)p; p += 8ull * n->nc;
    n->reg_d = (const uint32_t *)p; p += 4ull * n->nr;
    n->argoff = (const uint32_t *)p; p += 4ull * (n->no + 1ull);
    n->args = (const uint32_t *)p; p += 4ull * n->na;
    n->mem_words = (const uint32_t *)p; p += 4ull * n->nm;
    n->wport = (const uint32_t *)p; p += 16ull * n->nw;
    n->dom_period = (const uint32_t *)p; p += 4ull * n->nd;
    n->dom_phase = (const uint32_t *)p; p += 4ull * n->nd;
    n->in_w = p; p += n->ni;
    n->reg_w = p; p += n->nr;
    n->const_w = p; p += n->nc;
    n->code = p; p += n->no;
    n->width = p; p += n->no;
    n->p0 = p; p += n->no;
    n->p1 = p; p += n->no;
    n->mem_w = p; p += n->nm;
    n->reg_dom = n->nd ? p : NULL;
  }
  for (uint32_t d = 0; d < n->nd; d++) {
    uint32_t per = n->dom_period[d];
    if (per == 0 || per > (1u << 31) || (per & (per - 1)) != 0 || n->dom_phase[d] >= per) goto bad;
  }
  for (uint32_t r = 0; n->nd && r < n->nr; r++) if (n->reg_dom[r] >= n->nd) goto bad;
  n->reg_base = n->ni;
  n->const_base = n->ni + n->nr;
  n->op_base = n->ni + n->nr + n->nc;
  n->nsig = n->op_base + n->no;
  for (uint32_t i = 0; i < n->ni; i++) if (n->in_w[i] < 1 || n->in_w[i] > 64) goto bad;
  for (uint32_t i = 0; i < n->nr; i++) {
    if (n->reg_w[i] < 1 || n->reg_w[i] > 64 || n->reg_d[i] >= n->nsig) goto bad;
  }
  for (uint32_t i = 0; i < n->nc; i++) if (n->const_w[i] < 1 || n->const_w[i] > 64) goto bad;
  if (n->argoff[0] != 0 || n->argoff[n->no] != n->na) goto bad;
  n->mem_off = (uint64_t *)calloc(n->nm + 1, sizeof(uint64_t));
  for (uint32_t m = 0; m < n->nm; m++) {
    uint32_t w = n->mem_words[m];
    if (w == 0 || (w & (w - 1)) != 0 || n->mem_w[m] < 1 || n->mem_w[m] > 64) goto bad;
    n->mem_off[m + 1] = n->mem_off[m] + w;
  }
  n->mem_total = n->mem_off[n->nm];
  for (uint32_t k = 0; k < n->no; k++) {
    uint32_t c = n->code[k], w = n->width[k];
    uint32_t a0 = n->argoff[k], a1 = n->argoff[k + 1];
    if (a1 < a0 || w < 1 || w > 64 || c >= O_COUNT) goto bad;
    uint32_t cnt = a1 - a0;
    for (uint32_t j = a0; j < a1; j++) if (n->args[j] >= n->op_base + k) goto bad; /* topological */
    switch (c) {
      case O_AND: case O_OR: case O_XOR: case O_ADD: case O_MUL:
        if (cnt < 2) goto bad;
        break;
      case O_SUB: case O_DSHL: case O_DSHR: case O_CAT: case O_EQ: case O_NEQ: case O_LT:
      case O_LEQ: case O_GT: case O_GEQ:
        if (cnt != 2) goto bad;
        break;
      case O_MUX:
        if (cnt != 3) goto bad;
        break;
      case O_MUXCHAIN:
        if (cnt < 3 || (cnt & 1u) == 0) goto bad;
        break;
      case O_BITS:
        if (cnt != 1 || n->p0[k] < n->p1[k] || n->p0[k] > 63) goto bad;
        break;
      case O_ANDR:
        if (cnt != 1 || n->p0[k] < 1 || n->p0[k] > 64) goto bad;
        break;
      case O_MEMRD:
        if (cnt != 1 || (uint32_t)(n->p0[k] | (n->p1[k] << 8)) >= n->nm) goto bad;
        break;
      default:
        if (cnt != 1) goto bad;
        break;
    }
    if (c == O_CAT && (n->p0[k] < 1 || n->p0[k] > 64)) goto bad;
  }
  for (uint32_t p = 0; p < n->nw; p++) {
    const uint32_t *w = n->wport + 4ull * p;
    if (w[0] >= n->nm || w[1] >= n->nsig || w[2] >= n->nsig || w[3] >= n->nsig) goto bad;
  }
  return 0;
bad:
  onl_free(n);
  return -2;
}

/* One operation, written straight from its definition. */
static uint64_t eval_op(const onl *n, uint32_t k, const uint64_t *v, const uint64_t *mem) {
  const uint32_t *a = n->args + n->argoff[k];
  uint32_t cnt = n->argoff[k + 1] - n->argoff[k];
  unsigned p0 = n->p0[k], p1 = n->p1[k];
  uint64_t r = 0, x, y;
  switch (n->code[k]) {
    case O_COPY: r = v[a[0]]; break;
    case O_AND: r = v[a[0]]; for (uint32_t i = 1; i < cnt; i++) r &= v[a[i]]; break;
    case O_OR: r = v[a[0]]; for (uint32_t i = 1; i < cnt; i++) r |= v[a[i]]; break;
    case O_XOR: r = v[a[0]]; for (uint32_t i = 1; i < cnt; i++) r ^= v[a[i]]; break;
    case O_ADD: r = v[a[0]]; for (uint32_t i = 1; i < cnt; i++) r += v[a[i]]; break;
    case O_MUL: r = v[a[0]]; for (uint32_t i = 1; i < cnt; i++) r *= v[a[i]]; break;
    case O_NOT: r = ~v[a[0]]; break;
    case O_SUB: r = v[a[0]] - v[a[1]]; break;
    case O_SHL: r = p0 >= 64 ? 0 : v[a[0]] << p0; break;
    case O_SHR: r = p0 >= 64 ? 0 : v[a[0]] >> p0; break;
    case O_DSHL: x = v[a[0]]; y = v[a[1]]; r = y >= 64 ? 0 : x << y; break;
    case O_DSHR: x = v[a[0]]; y = v[a[1]]; r = y >= 64 ? 0 : x >> y; break;
    case O_BITS: r = (v[a[0]] >> p1) & mask_w(p0 - p1 + 1); break;
    case O_CAT: r = (p0 >= 64 ? 0 : v[a[0]] << p0) | v[a[1]]; break;
    case O_EQ: r = v[a[0]] == v[a[1]]; break;
    case O_NEQ: r = v[a[0]] != v[a[1]]; break;
    case O_LT: r = v[a[0]] < v[a[1]]; break;
    case O_LEQ: r = v[a[0]] <= v[a[1]]; break;
    case O_GT: r = v[a[0]] > v[a[1]]; break;
    case O_GEQ: r = v[a[0]] >= v[a[1]]; break;
    case O_MUX: r = (v[a[0]] & 1u) ? v[a[1]] : v[a[2]]; break;
    case O_ANDR: r = (v[a[0]] & mask_w(p0)) == mask_w(p0); break;
    case O_ORR: r = v[a[0]] != 0; break;
    case O_XORR: { x = v[a[0]]; unsigned c = 0; while (x) { c ^= (unsigned)(x & 1u); x >>= 1; } r = c; } break;
    case O_MEMRD: {
      uint32_t m = p0 | (p1 << 8);
      r = mem[n->mem_off[m] + (v[a[0]] & (uint64_t)(n->mem_words[m] - 1))];
    } break;
    case O_MUXCHAIN: {
      uint32_t pairs = (cnt - 1) / 2, i;
      r = v[a[cnt - 1]];
      for (i = 0; i < pairs; i++) {
        if (v[a[2 * i]] & 1u) { r = v[a[2 * i + 1]]; break; }
      }
    } break;
    default: r = 0; break;
  }
  return r & mask_w(n->width[k]);
}

typedef struct {
  const onl *n;
  uint32_t n_inst, i0, i1;
  uint64_t *vals, *mems;
  uint32_t *ticks;                      /* [n_inst] t of each instance (domains) */
  const uint32_t *cycles;
  int reset, stim_mode;
  uint64_t *xs; uint32_t xs_ld;
  const uint64_t *stim; uint32_t stim_ld, stim_cycles;
  const uint32_t *probe_sig; uint32_t n_probe; uint64_t *probe_out; uint32_t probe_cycles;
  int rc;
} job_t;

static void *run_range(void *arg) {
  job_t *j = (job_t *)arg;
  const onl *n = j->n;
  uint64_t *next = (uint64_t *)malloc(sizeof(uint64_t) * (n->nr ? n->nr : 1));
  for (uint32_t i = j->i0; i < j->i1; i++) {
    uint64_t *v = j->vals + (uint64_t)i * n->nsig;
    uint64_t *mem = j->mems + (uint64_t)i * n->mem_total;
    for (uint32_t c = 0; c < j->cycles[i]; c++) {
      /* 1. primary inputs */
      for (uint32_t q = 0; q < n->ni; q++) {
        uint64_t val = v[q];
        if (j->stim_mode == 1) {            /* xorshift64, Marsaglia 2003, shifts (13, 7, 17) */
          uint64_t x = j->xs[(uint64_t)q * j->xs_ld + i];
          x ^= x << 13;
          x ^= x >> 7;
          x ^= x << 17;
          j->xs[(uint64_t)q * j->xs_ld + i] = x;
          val = x;
        } else if (j->stim_mode == 2) {     /* explicit values [cycle][input][instance] */
          if (c >= j->stim_cycles) { j->rc = -1; goto out; }
          val = j->stim[((uint64_t)c * n->ni + q) * j->stim_ld + i];
        }
        v[q] = val & mask_w(n->in_w[q]);
      }
      /* 2. every operation, in topological order */
      for (uint32_t k = 0; k < n->no; k++) v[n->op_base + k] = eval_op(n, k, v, mem);
      /* 3. clock edge: next states from pre-edge values, memory writes, then commit */
      for (uint32_t r = 0; r < n->nr; r++) {
        if (j->reset) {
          next[r] = n->reg_init[r] & mask_w(n->reg_w[r]);
        } else if (n->nd && (uint32_t)(j->ticks[i] + n->dom_phase[n->reg_dom[r]]) %
                                    n->dom_period[n->reg_dom[r]] != 0) {
          next[r] = v[n->reg_base + r];     /* its domain does not tick this cycle */
        } else {
          next[r] = v[n->reg_d[r]] & mask_w(n->reg_w[r]);
        }
      }
      if (n->nd) j->ticks[i] = j->reset ? 0u : j->ticks[i] + 1u;
      for (uint32_t p = 0; p < n->nw; p++) {
        const uint32_t *w = n->wport + 4ull * p;
        if (v[w[1]] & 1u) {
          uint32_t m = w[0];
          mem[n->mem_off[m] + (v[w[2]] & (uint64_t)(n->mem_words[m] - 1))] =
              v[w[3]] & mask_w(n->mem_w[m]);
        }
      }
      for (uint32_t r = 0; r < n->nr; r++) v[n->reg_base + r] = next[r];
      /* probes: every signal's value at the end of the cycle */
      if (j->probe_out && c < j->probe_cycles) {
        for (uint32_t p = 0; p < j->n_probe; p++)
          j->probe_out[((uint64_t)c * j->n_probe + p) * j->n_inst + i] = v[j->probe_sig[p]];
      }
    }
  }
out:
  free(next);
  return NULL;
}

/* ------------------------------------------------------------------ API */

int oracle_sizes(const uint8_t *nl, size_t nb, uint64_t *out /* [n_signals, mem_words_total,
                 n_inputs, n_regs, n_consts, n_ops, n_mems, n_wports] */) {
  onl n;
  int rc = onl_parse(nl, nb, &n);
  if (rc) return rc;
  out[0] = n.nsig; out[1] = n.mem_total; out[2] = n.ni; out[3] = n.nr;
  out[4] = n.nc; out[5] = n.no; out[6] = n.nm; out[7] = n.nw;
  onl_free(&n);
  return 0;
}

/* vals: [n_inst][n_signals]; mems: [n_inst][mem_words_total].  Zeroes everything
 * and writes the constants. */
int oracle_init(const uint8_t *nl, size_t nb, uint32_t n_inst, uint64_t *vals, uint64_t *mems) {
  onl n;
  int rc = onl_parse(nl, nb, &n);
  if (rc) return rc;
  memset(vals, 0, sizeof(uint64_t) * (uint64_t)n_inst * n.nsig);
  if (n.mem_total) memset(mems, 0, sizeof(uint64_t) * (uint64_t)n_inst * n.mem_total);
  for (uint32_t i = 0; i < n_inst; i++)
    for (uint32_t c = 0; c < n.nc; c++)
      vals[(uint64_t)i * n.nsig + n.const_base + c] = n.const_value[c] & mask_w(n.const_w[c]);
  onl_free(&n);
  return 0;
}

/* Runs cycles[i] cycles on instance i; ticks [n_inst] (needed with clock
 * domains, else nullable) holds each instance's t and is updated.  stim_mode: 0 hold, 1 xorshift (xs is
 * [n_inputs][xs_ld], updated in place), 2 explicit values stim[cycle][input][stim_ld].
 * probe_out (nullable) receives [cycle][probe][n_inst] for cycle < probe_cycles.
 * Returns 0, -1 (bad argument) or -2 (format). */
int oracle_run(const uint8_t *nl, size_t nb, uint32_t n_inst, uint64_t *vals, uint64_t *mems,
               uint32_t *ticks, const uint32_t *cycles, int reset, int stim_mode, uint64_t *xs, uint32_t xs_ld,
               const uint64_t *stim, uint32_t stim_ld, uint32_t stim_cycles,
               const uint32_t *probe_sig, uint32_t n_probe, uint64_t *probe_out,
               uint32_t probe_cycles, int n_threads) {
  onl n;
  int rc = onl_parse(nl, nb, &n);
  if (rc) return rc;
  if ((stim_mode == 1 && !xs) || (stim_mode == 2 && !stim) || stim_mode < 0 || stim_mode > 2 ||
      (n.nd && !ticks)) {
    onl_free(&n);
    return -1;
  }
  for (uint32_t p = 0; p < n_probe; p++) if (probe_sig[p] >= n.nsig) { onl_free(&n); return -1; }
  if (n_threads < 1) n_threads = 1;
  if ((uint32_t)n_threads > n_inst) n_threads = n_inst ? (int)n_inst : 1;
  job_t *jobs = (job_t *)calloc((size_t)n_threads, sizeof(job_t));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int t = 0; t < n_threads; t++) {
    job_t *j = &jobs[t];
    j->n = &n; j->n_inst = n_inst;
    j->i0 = (uint32_t)((uint64_t)n_inst * t / n_threads);
    j->i1 = (uint32_t)((uint64_t)n_inst * (t + 1) / n_threads);
    j->vals = vals; j->mems = mems; j->ticks = ticks; j->cycles = cycles; j->reset = reset;
    j->stim_mode = stim_mode; j->xs = xs; j->xs_ld = xs_ld;
    j->stim = stim; j->stim_ld = stim_ld; j->stim_cycles = stim_cycles;
    j->probe_sig = probe_sig; j->n_probe = n_probe; j->probe_out = probe_out;
    j->probe_cycles = probe_cycles;
  }
  if (n_threads == 1) {
    run_range(&jobs[0]);
  } else {
    for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, run_range, &jobs[t]);
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
  }
  for (int t = 0; t < n_threads; t++) if (jobs[t].rc) rc = jobs[t].rc;
  free(jobs);
  free(th);
  onl_free(&n);
  return rc;
}

/* Single-operation evaluation for the per-opcode pins: builds nothing, just
 * applies the definition above to explicit operand values. */
uint64_t oracle_eval_one(uint32_t code, uint32_t width, uint32_t p0, uint32_t p1,
                         const uint64_t *operands, uint32_t n_operands) {
  uint32_t argoff[2] = {0, n_operands};
  uint32_t args[64];
  uint8_t c = (uint8_t)code, w = (uint8_t)width, q0 = (uint8_t)p0, q1 = (uint8_t)p1;
  onl n;
  memset(&n, 0, sizeof(n));
  if (n_operands > 64) return 0;
  for (uint32_t i = 0; i < n_operands; i++) args[i] = i;
  n.argoff = argoff; n.args = args; n.code = &c; n.width = &w; n.p0 = &q0; n.p1 = &q1;
  return eval_op(&n, 0, operands, NULL);
}

/* Batch form of oracle_eval_one: operands is [n][k] (k operands per row). */
void oracle_eval_batch(uint32_t code, uint32_t width, uint32_t p0, uint32_t p1,
                       const uint64_t *operands, uint32_t k, uint64_t n, uint64_t *out) {
  for (uint64_t i = 0; i < n; i++) out[i] = oracle_eval_one(code, width, p0, p1, operands + i * k, k);
}
