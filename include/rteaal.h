/* rteaal.h -- C ABI of librteaal.so: GPU (sm_103a) cycle-accurate RTL simulation
 * as a cascade of extended Einsums (RTeAAL Sim, arXiv 2601.18140).
 *
 * What one cycle computes (Sec. 4, Cascade 1 of the paper, loop order of
 * Alg. 3 / Alg. 4):
 *   for each layer i (iterative rank I):
 *     OI       = LI_i . OIM_i                (gather the operands named by the mask)
 *     LO_i     = op_u[n], then op_r[n] folded in ascending O order
 *     LO_sel_i = op_s[n] over the O-fiber    (select operations, e.g. mux)
 *     LI_{i+1} = LO_i | LO_sel_i
 *   then every register commits its next state at the clock edge (Sec. 2.1,
 *   Fig. 1), and the testbench drives the primary inputs at the cycle boundary
 *   (Sec. 6.2, "Host-DUT Communication").
 *
 * Device form.  Identity operations are elided by giving every signal one
 * global row (Sec. 4.3): LI / LO of every layer are views of one state array,
 * so that LI_{i+1} <- LO_i moves no data and is only a barrier.  State layout
 * ("compact"): one row per slot, lane-minor (lane = stimulus instance); a row
 * holds 1, 2, 4 or 8 bytes per lane for signal widths up to 8, 16, 32, 64
 * (width class k = 0..3); the rows of class 3 come first, then 2, 1, 0; inside
 * a class, pool rows (inputs, registers, constants in signal order) precede op
 * rows (slot order).  A row's per-lane byte offset o is the sum of the bytes
 * per lane of all rows before it; element (row, lane) of an n-lane state is the
 * little-endian integer of 1 << k bytes at byte o * n + (lane << k).  OIM is lowered
 * to per-layer operand lists whose operations are grouped by (opcode, width)
 * -- the swizzled [I, N, S, O, R] order of the NU kernel (Sec. 5.2) -- with the
 * S coordinates implicit (the outputs of a layer occupy consecutive slots) and
 * the N / O payloads implied by the opcode (Sec. 5.1, "Compressing the OIM").
 *
 * ------------------------------------------------------------------------
 * Netlist format "RTLN" version 1 (input of rteaal_design_load)
 * ------------------------------------------------------------------------
 * Little-endian.  Header: 10 x u32
 *     magic 0x4E4C5452, version 1, n_inputs, n_regs, n_consts, n_ops,
 *     n_mems, n_wports, n_args, n_domains (0: one clock)
 * then, in this order (the [..] parts only when n_domains > 0):
 *     u64 reg_init[n_regs]        u64 const_value[n_consts]
 *     u32 reg_d[n_regs]           u32 op_argoff[n_ops+1]   u32 args[n_args]
 *     u32 mem_words[n_mems]       u32 wport[n_wports][4] = {mem, en, addr, data}
 *     [u32 domain_period[n_domains]   u32 domain_phase[n_domains]]
 *     u8 input_width[n_inputs]    u8 reg_width[n_regs]     u8 const_width[n_consts]
 *     u8 op_code[n_ops]  u8 op_width[n_ops]  u8 op_p0[n_ops]  u8 op_p1[n_ops]
 *     u8 mem_width[n_mems]        [u8 reg_domain[n_regs]]
 * Signal ids: [0, n_inputs) inputs, then registers (their Q), then constants,
 * then op outputs in topological order (every operand id < the op's own id).
 * Op k's operands are args[op_argoff[k] .. op_argoff[k+1]) in O order.
 *
 * Clock domains (Sec. 6.2 "Multiple Clock Domains"; the rule is a reading):
 * domain d has a period p (a power of two <= 2^31, in base-clock cycles) and a
 * phase f < p; every register names its domain (at most 256).  Each instance
 * counts t, the non-reset cycles since its last reset cycle; at the edge of a
 * non-reset cycle a register of domain (p, f) takes its next state only if
 * (t + f) mod p == 0, else it holds; a reset cycle resets every register and t.
 * Memory write ports run on the base clock.  The library lowers the domains to
 * one clock (a hidden 32-bit cycle counter and a hold mux per register of a
 * slower domain), so every kernel form and option supports them; the hidden
 * signals have no id.
 *
 * Value domain (reading: the paper claims support for every FIRRTL primitive
 * operation without defining any): unsigned only; every signal has a width w in 1..64 and
 * is stored zero-extended in 64 bits, always masked to w.  mask(w) = 2^w - 1.
 * Every op result is masked to the op's width.  Opcodes (u8):
 *   0 COPY a            1 AND a,b,...   2 OR a,b,...   3 XOR a,b,...  (fold in O order)
 *   4 NOT ~a            5 ADD a,b,...   6 SUB a-b      7 MUL a*b*... (all mod 2^64)
 *   8 SHL a<<p0         9 SHR a>>p0    10 DSHL a<<b   11 DSHR a>>b   (amount >= 64 -> 0)
 *  12 BITS (a>>p1) & mask(p0-p1+1)  (hi = p0 >= lo = p1, hi <= 63)
 *  13 CAT (a<<p0) | b   (p0 = width of b, 1..64; o0 is the high part)
 *  14 EQ 15 NEQ 16 LT 17 LEQ 18 GT 19 GEQ   unsigned, result 0/1
 *  20 MUX  (sel & 1) ? o1 : o2   (O=0 is the selector; App. A; FIRRTL order)
 *  21 ANDR (a & mask(p0)) == mask(p0) (p0 = operand width)  22 ORR a != 0
 *  23 XORR parity of a           24 MEMRD mem[p0 | p1<<8][a & (words-1)]
 *  25 MUXCHAIN s0,v0,s1,v1,...,default: v_i of the first s_i with bit 0 set,
 *     else default (operator fusion of mux chains, App. B.1)
 * Classes (Cascade 1): op_u = unary ops (COPY NOT SHL SHR BITS ANDR ORR XORR
 * MEMRD); op_r = reducible ops (the binary ones, folded in O order); op_s =
 * select ops (MUX MUXCHAIN).
 * Clock edge (reading; the paper has no reset or memories): Q <- (reset ?
 * init : value(D)) & mask(w_Q).  Memories hold words x mem_width bits, are
 * zero at rteaal_sim_create and untouched by reset; MEMRD sees the pre-edge
 * contents; at the edge each write port, in port order, writes data &
 * mask(mem_width) to addr & (words-1) when en & 1 (a later port wins).
 * words must be a power of two.
 * One cycle: (1) drive inputs (value & mask(w_in)); (2) all ops; (3) edge.
 * ------------------------------------------------------------------------ */
#ifndef RTEAAL_H
#define RTEAAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rteaal_design rteaal_design; /* opaque, immutable after load   */
typedef struct rteaal_sim rteaal_sim;       /* opaque, device state of a batch */

/* Every entry point returns one of these (0 = success).  No C++ exception
 * crosses the ABI.  On failure rteaal_last_error() describes the cause. */
enum {
  RTEAAL_OK = 0,
  RTEAAL_E_INVALID = -1,     /* bad argument (null pointer, range, mode)            */
  RTEAAL_E_FORMAT = -2,      /* netlist bytes malformed or violate the rules above  */
  RTEAAL_E_NOMEM = -3,       /* device allocation failed / footprint refused        */
  RTEAAL_E_CUDA = -4,        /* a CUDA call failed (message has the CUDA error)     */
  RTEAAL_E_TIMEOUT = -5,     /* a bounded device-side wait gave up (grid barrier)   */
  RTEAAL_E_BUSY = -6,        /* object still in use (e.g. design with live sims)    */
  RTEAAL_E_UNSUPPORTED = -7  /* valid request this build cannot run                 */
};

/* Device-memory provider.  alloc returns a device pointer aligned to >= 256
 * bytes or NULL; free releases it.  NULL provider = cudaMalloc / cudaFree.
 * The Python binding passes PyTorch's caching allocator here. */
typedef struct {
  void *(*alloc)(size_t bytes, void *ctx);
  void (*free)(void *ptr, size_t bytes, void *ctx);
  void *ctx;
} rteaal_allocator;

/* ---------------------------------------------------------------- design */
typedef struct {
  const rteaal_allocator *allocator; /* nullable */
  int device;                        /* CUDA ordinal; < 0 = current device */
  /* Operator fusion (App. B.1, mux-chain extraction): a MUX whose false operand
   * is another MUX read nowhere else and at least as wide is absorbed, and the
   * chain is evaluated as one MUXCHAIN.  Absorbed signals are not computed:
   * reading or probing them is refused (E_INVALID), as the paper disables
   * signal-eliminating optimizations when every signal must stay visible. */
  int fuse_mux_chains;
} rteaal_load_opts;

typedef struct {
  uint32_t n_signals, n_inputs, n_regs, n_consts, n_ops, n_mems, n_wports;
  uint32_t n_layers;         /* levels after levelisation (Sec. 4.2)            */
  uint32_t n_groups;         /* non-empty (layer, opcode, width) groups          */
  uint32_t n_slots;          /* state rows per lane (signals + inserted copies)  */
  uint32_t n_lowered_ops;    /* ops evaluated per cycle incl. inserted copies    */
  uint32_t max_layer_ops;
  uint64_t op_operands;      /* sum of operand counts over the n_ops netlist ops */
  uint64_t mem_words_total;  /* words of all memories of one lane               */
  uint64_t metadata_bytes;   /* device bytes owned by the design                */
  uint64_t state_bytes_per_lane; /* compact state bytes of one lane (see layout) */
  uint32_t n_fused;          /* muxes absorbed by operator fusion               */
} rteaal_design_stats;

/* Parse, validate, levelise, group by (opcode, width) and upload the lowered
 * operand lists.  netlist: host bytes (copied; caller keeps ownership).
 * opts nullable.  *out receives a handle owned by the caller, released with
 * rteaal_design_free.  Errors: E_INVALID, E_FORMAT, E_NOMEM, E_CUDA. */
int rteaal_design_load(const void *netlist, size_t nbytes, const rteaal_load_opts *opts,
                       rteaal_design **out);
/* Figures of a loaded design (the netlist's counts and its lowering: layers
 * of Sec. 4.2, (layer, opcode, width) groups, compact state size, device bytes
 * of the lowered operand lists).  out: caller-owned.  Errors: E_INVALID. */
int rteaal_design_info(const rteaal_design *design, rteaal_design_stats *out);
/* Which signals hold a row of the state: present[i] = 1 for signal i that can
 * be read, written and probed, 0 for a mux absorbed by operator fusion.
 * present: host array of n_signals bytes (caller-owned); n_signals must equal
 * the design's signal count.  Errors: E_INVALID. */
int rteaal_design_signals(const rteaal_design *design, uint8_t *present, uint64_t n_signals);
/* Generate and compile the design-specialised kernel (RTEAAL_KERNEL_SPECIALIZED)
 * now instead of at the first configure that asks for it; *compile_us
 * (nullable) receives the generation + compile time of the first call (the
 * kernel is kept with the design).  Errors: E_UNSUPPORTED (too many ops),
 * E_CUDA (compile or load failure; the message holds the compiler log). */
int rteaal_design_specialize(rteaal_design *design, uint64_t *compile_us);
/* ---------------------------------------------------------------- host-only inspection
 * The calls below (up to rteaal_design_specialized_source) parse and lower a netlist
 * on the host, touch no device and keep nothing: they expose what the kernels will
 * execute so that it can be checked without a GPU. */
/* The lowering alone, on the host (no device is touched, nothing is kept):
 * parse, lower clock domains, fuse (opts->fuse_mux_chains), levelise (Sec. 4.2:
 * an op's layer is one more than the deepest of its operands; inputs,
 * registers and constants are layer 0) and group, exactly as
 * rteaal_design_load does.  *out receives the figures rteaal_design_info would
 * report for the loaded design, except metadata_bytes = 0 (nothing uploaded).
 * layer_ops (nullable, caller-owned host array of max_layers entries) receives
 * the lowered op count of layers 1, 2, ... (first max_layers of them).
 * opts nullable; its allocator and device are ignored.
 * Errors: E_INVALID (null netlist or out), E_FORMAT (as rteaal_design_load). */
int rteaal_design_lower(const void *netlist, size_t nbytes, const rteaal_load_opts *opts,
                        rteaal_design_stats *out, uint32_t *layer_ops, uint32_t max_layers);
/* The one-clock netlist the library simulates for a netlist with clock domains
 * (Sec. 6.2 "Multiple Clock Domains", reading in the format notes above): a
 * hidden 32-bit cycle counter t (a register after the caller's registers), per
 * slower domain an enable (t + phase) & (period - 1) == 0, and per register of
 * such a domain a hold mux; without domains, the netlist itself.  Host only.
 * out (nullable, caller-owned, capacity bytes) receives its RTLN bytes and
 * *out_bytes their count (call with out = NULL to size the buffer).  user2x
 * (nullable, caller-owned, n_user = the netlist's signal count) receives, for
 * every caller signal, its id in the one-clock netlist.
 * Errors: E_INVALID (null netlist or out_bytes, capacity or n_user too small or
 * wrong), E_FORMAT (as rteaal_design_load). */
int rteaal_design_single_clock(const void *netlist, size_t nbytes, void *out, size_t capacity,
                               size_t *out_bytes, uint32_t *user2x, uint64_t n_user);
/* The lowered design as the kernels execute it, written back as a netlist
 * (host only): one signal per state row -- inputs, registers (with the hidden
 * cycle counter of clock domains), constants, then one op per descriptor in
 * the lowered order (layer by layer, Sec. 4.2; grouped by opcode and width),
 * each decoded from its descriptor: fused mux chains as MUXCHAIN, the copies
 * the clock edge reads as COPY; registers and write ports from the edge
 * tables.  Simulating it gives every surviving signal the value the design
 * gives it.  out / capacity / out_bytes as rteaal_design_single_clock;
 * user2sig (nullable, caller-owned, n_user = the netlist's signal count)
 * receives each caller signal's id there, 0xFFFFFFFF for a mux absorbed by
 * fusion.  opts nullable (only fuse_mux_chains is read).
 * Errors: E_INVALID, E_FORMAT (as rteaal_design_load). */
int rteaal_design_lowered_netlist(const void *netlist, size_t nbytes, const rteaal_load_opts *opts, void *out,
                                  size_t capacity, size_t *out_bytes, uint32_t *user2sig, uint64_t n_user);
/* The compact layout of the lowered design (host only): refs (caller-owned,
 * n_rows = the lowered design's row count, i.e. the signal count of
 * rteaal_design_lowered_netlist, whose signal ids index it) receives every
 * row's reference, width class k << 30 | per-lane byte offset (layout in the
 * notes at the top of this file).  opts nullable (only fuse_mux_chains is
 * read).  Errors: E_INVALID (null argument, wrong n_rows), E_FORMAT. */
int rteaal_design_rows(const void *netlist, size_t nbytes, const rteaal_load_opts *opts, uint32_t *refs,
                       uint64_t n_rows);
/* The FLOW form's tables for the lowered design (host only; the tables the
 * library uploads at a sim's first FLOW step).  Rows are counted in layout
 * order: class-3 rows first, then 2, 1, 0, each class in reference order.
 * op (nullable, caller-owned, 8 uint32 per lowered op, in slot order): rows of
 * operands a, b, c -- bit 31 set on a row that an op writes in the cycle, whose
 * stamp the item waits for (Cascade 1's LI_{i+1} <- LO_i step as a per-operand
 * wait); 0 for an absent operand and for ops with more than three operands --
 * then the output's row, ctl, the output's reference, and for ops with more
 * than three operands the offset and count of their operand rows in ext
 * (nullable, caller-owned, *n_ext entries, flagged the same way).  pool
 * (nullable, caller-owned, 2 uint32 per row): {reference, row} of every input,
 * register and constant, in that order.  *n_op, *n_ext, *n_pool: on entry the
 * capacities of the arrays given (checked), on return the counts; call with
 * null arrays to size them.  opts nullable (only fuse_mux_chains is read).
 * Errors: E_INVALID (null count pointer, wrong capacity), E_FORMAT. */
int rteaal_design_flow_tables(const void *netlist, size_t nbytes, const rteaal_load_opts *opts, uint32_t *op,
                              uint64_t *n_op, uint32_t *ext, uint64_t *n_ext, uint32_t *pool, uint64_t *n_pool);
/* The design-specialised kernel's generation and NVRTC compile for sm_103a
 * alone, on the host (no device is touched, nothing is kept): checks that a
 * netlist's straight-line kernel (Sec. 5.2, unrolled S rank and inlined
 * tensors) compiles.  cubin_bytes / compile_us (nullable) receive the size of
 * the compiled image and the generation + compile time.  opts nullable (only
 * fuse_mux_chains is read).  Errors: E_INVALID, E_FORMAT, E_UNSUPPORTED (too
 * many ops), E_CUDA (compile failure; the message holds the compiler log). */
int rteaal_design_specialize_host(const void *netlist, size_t nbytes, const rteaal_load_opts *opts,
                                  uint64_t *cubin_bytes, uint64_t *compile_us);
/* The design-specialised kernel's CUDA source text (the kernel rteaal_spec:
 * one thread per lane, every signal a local, one statement per op), as
 * generated for the lowered design; host only.  out (nullable, caller-owned,
 * capacity bytes, not NUL-terminated) receives the text and *out_bytes its
 * length (call with out = NULL to size the buffer).  opts nullable (only
 * fuse_mux_chains is read).  Errors: E_INVALID, E_FORMAT. */
int rteaal_design_specialized_source(const void *netlist, size_t nbytes, const rteaal_load_opts *opts, char *out,
                                     size_t capacity, size_t *out_bytes);
/* Returns E_BUSY (and frees nothing) while sims created from it are alive. */
int rteaal_design_free(rteaal_design *design);

/* ---------------------------------------------------------------- simulation */
enum {
  RTEAAL_KERNEL_AUTO = 0,   /* TILE when lanes >= 64, else LAYER; GRID with activity */
  RTEAAL_KERNEL_LAYER = 1,  /* plain form: one launch per layer per cycle          */
  RTEAAL_KERNEL_TILE = 2,   /* persistent: a CTA walks all layers and cycles of an
                               instance tile, CTA barrier between layers           */
  RTEAAL_KERNEL_GRID = 3,   /* persistent cooperative: the whole grid walks all
                               layers, bounded grid barrier between layers         */
  RTEAAL_KERNEL_LAYER_GRAPH = 4, /* plain form with the cycle loop as a CUDA graph */
  RTEAAL_KERNEL_STREAM = 5, /* persistent cooperative, one CTA per SM: a producer
                               warp streams each op's operand rows into a
                               shared-memory ring with bulk copies (TMA engine,
                               mbarriers), consumer warps compute from it; needs a
                               multiple of 128 lanes                              */
  RTEAAL_KERNEL_CLUSTER = 7,  /* thread-block clusters (up to 16 CTAs, one per SM)
                               each own a tile of tile_lanes lanes and walk every
                               layer of every cycle of it with the hardware
                               cluster barrier between layers (for few lanes:
                               one instance, the tail of a job)                   */
  RTEAAL_KERNEL_FLOW = 8,   /* persistent cooperative, one lane per item, no barrier
                               between layers (Cascade 1's LI_{i+1} <- LO_i step
                               as a per-operand wait): every result is also written
                               to a word holding it next to the cycle's stamp, and
                               an item waits (bounded) until the operands it reads
                               carry this cycle's stamp; grid barriers only around
                               the stimulus and the clock edge.  For few lanes (one
                               instance); its stamped words take 16 bytes per row
                               and lane of extra device memory, allocated at the
                               first FLOW step.  Error word bit 8: a wait gave up */
  RTEAAL_KERNEL_SPECIALIZED = 6 /* design-specialised (Sec. 5.2 SU / TI on the GPU):
                               the op list unrolled into straight-line code compiled
                               at run time (NVRTC), every signal a local variable,
                               one thread per instance for all cycles of a step;
                               state rows read once and written once per step.
                               Probes: LAST only.  Designs up to 16,384 ops (the
                               compile time grows superlinearly with the length). */
};

typedef struct {
  const rteaal_allocator *allocator; /* nullable */
  /* host [n_instances], nullable: expected cycle counts.  Lanes are ordered by
   * descending count so that instances of a tile retire together (uneven
   * cycle counts); lane order never changes the results. */
  const uint32_t *expected_cycles;
  /* host [n_inputs][n_instances], nullable: initial xorshift64 states for
   * RTEAAL_STIM_XORSHIFT (copied).  A zero state stays zero. */
  const uint64_t *xorshift_seed;
  int kernel;              /* RTEAAL_KERNEL_*                                   */
  uint32_t tile_lanes;     /* TILE: lanes per tile (power of two <= 64), 0 auto;
                              CLUSTER: lanes per cluster tile; FLOW: items a warp
                              takes per layer (1..32, 0 = 8)                     */
  uint32_t threads;        /* threads per CTA (multiple of 32, <= 1024), 0 auto */
  uint32_t ctas_per_sm;    /* TILE / GRID residency target, 0 auto              */
  uint32_t unroll;         /* operations in flight per thread (1, 2, 4), 0 auto */
  uint32_t lanes_per_thread; /* lanes (instances) per thread per op (1, 2, 4, 8), 0 auto */
  /* Activity-aware evaluation (App. B's cascade-level optimisation that leaves
   * out partitions whose inputs did not change, at the finest grain): the sim
   * keeps, per row and 128-lane chunk, the last cycle in which the row changed
   * in any lane of the chunk; an op is evaluated for a chunk only if one of its
   * operands changed there in the current cycle (memory reads always), and its
   * result is stored only if it differs.  Exact -- results never depend on it.
   * GRID kernel only (configure refuses the others: E_UNSUPPORTED); costs one
   * byte of device memory per row and chunk.  Fixed at creation. */
  int activity;
  uint32_t cluster_ctas;   /* CLUSTER: CTAs per cluster (2..16), 0 auto          */
  /* CLUSTER with one tile of at most 64 lanes: keep the whole state in the
   * cluster's distributed shared memory for the length of a step (0: when it
   * fits, 1: required -- E_UNSUPPORTED if it does not fit, -1: never). */
  int cluster_resident;
} rteaal_sim_opts;

typedef struct {
  uint32_t n_instances, n_lanes; /* n_lanes = padded lane count of the state    */
  uint64_t device_bytes;         /* state + memories + stimulus + scratch        */
  int kernel;                    /* kernel chosen                                */
  uint32_t tile_lanes, threads, ctas_per_sm, unroll, grid;
  uint32_t lanes_per_thread;
  int activity;                  /* activity-aware evaluation on                  */
  uint32_t last_span;            /* lanes the last rteaal_step visited (live prefix) */
  uint32_t last_grid;            /* CTAs of the last GRID launch (0: none yet)    */
  uint32_t cluster_ctas;         /* CLUSTER: CTAs per cluster                     */
  int cluster_resident;          /* CLUSTER: state kept in distributed shared memory */
} rteaal_sim_stats;

/* Allocates and zero-initialises the state of n_instances (>= 1) independent
 * instances -- LI / LO of every layer as one global row per signal (identity
 * elision, Sec. 4.3), one lane per stimulus instance -- and writes the constants.  Registers are 0 until a reset cycle.
 * design must outlive the sim.  Errors: E_INVALID, E_NOMEM, E_CUDA. */
int rteaal_sim_create(const rteaal_design *design, uint32_t n_instances,
                      const rteaal_sim_opts *opts, rteaal_sim **out);
/* Instance / lane counts, device bytes and the launch configuration in use.
 * out: caller-owned.  Errors: E_INVALID. */
int rteaal_sim_info(const rteaal_sim *sim, rteaal_sim_stats *out);
/* Waits for the device, then frees the sim's device memory (NULL: no-op). */
void rteaal_sim_destroy(rteaal_sim *sim);

/* Change the launch configuration (kernel, tile_lanes, threads, ctas_per_sm,
 * unroll, lanes_per_thread, cluster_ctas, cluster_resident of opts; the other
 * fields are ignored).  Results never depend on it.
 * Errors: E_INVALID, E_UNSUPPORTED (no compiled variant). */
int rteaal_sim_configure(rteaal_sim *sim, const rteaal_sim_opts *opts);

typedef struct {
  int kernel;
  uint32_t tile_lanes, threads, ctas_per_sm, unroll, grid, lanes_per_thread;  /* CLUSTER:
                                    ctas_per_sm holds the CTAs per cluster */
  float ms;                      /* device time of one trial step                 */
} rteaal_tune_trial;

/* Autotuner: times every candidate launch configuration of the kernels in
 * kernel_mask (bit 1 << RTEAAL_KERNEL_*, 0 = TILE|GRID|STREAM, or
 * LAYER|GRID|CLUSTER|FLOW for fewer than 64 lanes) on this sim, one warm-up and one timed step of
 * cycles_per_trial cycles each, keeps the fastest, and restores the state,
 * memories and stimulus states exactly (device-to-device snapshot: needs
 * free device memory equal to the sim's state).  trials (nullable) receives
 * up to max_trials results; *n_trials (nullable) the number run.
 * Synchronises stream.  Errors: E_NOMEM (no room for the snapshot), E_CUDA. */
int rteaal_sim_autotune(rteaal_sim *sim, uint32_t cycles_per_trial, uint32_t kernel_mask,
                        rteaal_tune_trial *trials, uint32_t max_trials, uint32_t *n_trials,
                        void *stream);

/* Activity-aware sims: (op, 128-lane chunk) items evaluated and skipped since
 * creation.  Synchronises stream.  Errors: E_INVALID. */
int rteaal_sim_activity(rteaal_sim *sim, uint64_t *evaluated, uint64_t *skipped, void *stream);

/* Bytes of device memory rteaal_sim_create would take (footprint admission).
 * Steps in the FLOW kernel add, at their first launch, 16 bytes per row and
 * padded lane (the stamped words) and 32 bytes per op (their descriptors). */
uint64_t rteaal_sim_footprint(const rteaal_design *design, uint32_t n_instances);

typedef struct {
  uint64_t uniform;              /* cycles for every instance if per_instance is NULL */
  const uint32_t *per_instance;  /* host [n_instances], nullable (uneven cycles)      */
  /* host [n_instances], nullable: the first r[i] cycles of this call are reset
   * cycles for instance i (RTEAAL_STEP_RESET makes every cycle of every
   * instance a reset cycle).  Lets one instance reset while others run. */
  const uint32_t *reset_per_instance;
} rteaal_cycles;

enum { RTEAAL_STIM_HOLD = 0, RTEAAL_STIM_XORSHIFT = 1, RTEAAL_STIM_BUFFER = 2 };
typedef struct {
  int mode;
  /* BUFFER: [cycles][n_inputs][n_instances] values (masked on use), instance
   * order = user order, cycle index relative to the step.  Device pointer,
   * or host pointer when values_on_host (copied inside the call; pinned
   * memory makes the copy asynchronous). */
  const uint64_t *values;
  int values_on_host;
} rteaal_stimulus;

enum { RTEAAL_PROBE_LAST = 0, RTEAAL_PROBE_EVERY = 1, RTEAAL_PROBE_CHANGES = 2 };

/* One waveform event (RTEAAL_PROBE_CHANGES): probe `probe` of instance
 * `instance` took `value` at the end of cycle `cycle` (cycle index relative to
 * the step) and that differs from its value at the end of the previous cycle
 * (for cycle 0: its value when the step began) -- waveform generation, Sec. 6.2,
 * which keeps a value only when it changes. */
typedef struct {
  uint32_t cycle, probe, instance, pad;
  uint64_t value;
} rteaal_change;

typedef struct {
  const uint32_t *signals;  /* host [n] signal ids */
  uint32_t n;
  int mode;                 /* LAST: out [n][n_instances] after the step;
                               EVERY: out [cycles][n][n_instances], row c written
                               for instances that ran cycle c (end-of-cycle values);
                               CHANGES: out = rteaal_change[capacity], unordered */
  uint64_t *out;            /* device pointer, or host if out_on_host          */
  int out_on_host;          /* host: copied back and synchronised in the call  */
  uint64_t capacity;        /* CHANGES: records that fit in out                */
  uint64_t *count;          /* CHANGES: host, receives the number of changes
                               (more than capacity: the excess was dropped);
                               the call synchronises                           */
} rteaal_probes;

enum { RTEAAL_STEP_RESET = 1 };

/* Advance every instance by its cycle count (0 allowed): per cycle, inputs
 * (Sec. 6.2 "Host--DUT Communication"), every layer of Cascade 1 in order
 * (Sec. 4.2, Alg. 3 / Alg. 4), then the register commit (Sec. 2.1, Fig. 1);
 * uneven counts are the iterative rank of Alg. 1 applied per instance.
 * Only lanes up to the last one with a nonzero count are visited (lanes are
 * ordered by expected_cycles, so finished instances cost nothing; a frozen
 * instance is never written).  flags & RESET makes
 * every cycle of the call a reset cycle.  Work is enqueued on stream (a
 * cudaStream_t; NULL = legacy default stream) and is asynchronous unless a
 * host buffer is involved.  Caller-owned device buffers must stay valid until
 * the stream reaches the end of the step.  Errors: E_INVALID, E_CUDA,
 * E_TIMEOUT (reported by this or the next call on the sim), E_UNSUPPORTED. */
int rteaal_step(rteaal_sim *sim, const rteaal_cycles *cycles, const rteaal_stimulus *stimulus,
                const rteaal_probes *probes /* nullable */, uint32_t flags, void *stream);

/* Return instances [inst_begin, inst_begin + n_inst) to the state of a fresh
 * sim -- every signal 0 except constants, memories 0 -- and set their
 * xorshift64 states from host [n_inputs][n_inst] (nullable: all 0).  Other
 * instances are untouched (a serving loop reuses freed instances this way).
 * Enqueued on stream; the seed buffer is copied before return. */
int rteaal_sim_reset_lanes(rteaal_sim *sim, uint32_t inst_begin, uint32_t n_inst,
                           const uint64_t *xorshift_seed, void *stream);

/* Blocks until the sim's work on stream is done; returns any pending error. */
int rteaal_sync(rteaal_sim *sim, void *stream);

/* Copy signal values (rows of LI / LO, Sec. 4.1; register Q values, Sec. 2.1)
 * of instances [inst_begin, inst_begin + n_inst) to / from host memory laid out [n][n_inst] (caller-owned, any host memory; values
 * zero-extended, writes masked to each signal's width).  signals: host array of
 * n signal ids (caller-owned).  Synchronises stream.  Writing a constant
 * changes it for the rest of the simulation (checkpoint restore).  Errors:
 * E_INVALID (null sim or buffer, instance range beyond n_instances, signal id
 * out of range or fused away), E_NOMEM (device staging buffer), E_CUDA. */
int rteaal_state_read(rteaal_sim *sim, const uint32_t *signals, uint32_t n, uint32_t inst_begin,
                      uint32_t n_inst, uint64_t *host_out, void *stream);
int rteaal_state_write(rteaal_sim *sim, const uint32_t *signals, uint32_t n, uint32_t inst_begin,
                       uint32_t n_inst, const uint64_t *host_in, void *stream);
/* Memory words of all memories (memory-major, word order): host buffer
 * [mem_words_total][n_inst] uint64 (caller-owned); written words are stored
 * as given (the caller keeps them within mem_width).  Synchronises stream.
 * Errors as rteaal_state_read. */
int rteaal_mem_read(rteaal_sim *sim, uint32_t inst_begin, uint32_t n_inst, uint64_t *host_out,
                    void *stream);
int rteaal_mem_write(rteaal_sim *sim, uint32_t inst_begin, uint32_t n_inst, const uint64_t *host_in,
                     void *stream);
/* xorshift64 stimulus states (Sec. 6.2 testbench; Marsaglia 2003): host buffer
 * [n_inputs][n_inst] uint64 (caller-owned); writing them replays a stimulus
 * from a checkpoint.  Synchronises stream.  Errors as rteaal_state_read. */
int rteaal_stim_state_read(rteaal_sim *sim, uint32_t inst_begin, uint32_t n_inst,
                           uint64_t *host_out, void *stream);
int rteaal_stim_state_write(rteaal_sim *sim, uint32_t inst_begin, uint32_t n_inst,
                            const uint64_t *host_in, void *stream);

/* ---------------------------------------------------------------- allocation-free step
 * No counterpart in the paper.  Some callers cannot allocate device memory at
 * all -- a host process whose device memory is owned by another allocator or
 * framework that forbids cudaMalloc / cudaFree from libraries, or that has
 * already handed out every byte.  For them this entry point runs the
 * persistent grid form over buffers they own and allocates nothing: no
 * cudaMalloc / cudaFree and no allocating library routine.  Its scratch (grid
 * barrier words, error word, per-lane cycle budgets) is a file-scope device
 * array sized for RTEAAL_STATIC_MAX_LANES lanes (about 256 KB), which every GPU
 * that loads the library holds until the process exits.
 *
 * Buffers (caller-owned device memory, lane = instance, identity order):
 *   state state_bytes_per_lane * n_lanes bytes in the compact layout above
 *         (constants' rows must hold their values)
 *   mem   [mem_words_total][n_lanes] uint64 (nullable without memories)
 *   xs    [n_inputs][n_lanes] uint64 xorshift64 states (nullable unless XORSHIFT)
 * Slot order of op rows (the layout's row order; rteaal_design_rows and
 * rteaal_design_lowered_netlist report it for a given netlist): by level;
 * inside a level, ops with at most three operands before the others; among
 * those, narrow ops before wide ones (narrow: the result and every operand at
 * most 32 bits wide, and the op is not MEMRD, not BITS with hi >= 32, not ANDR
 * over more than 32 bits); then (opcode, width); then netlist order.  A
 * register D or write-port signal that is not an op output gets a COPY op on
 * level 1, ordered after the netlist's own ops of the same key.  16-byte
 * aligned buffers with an even n_lanes use two lanes per thread, otherwise one.
 * The bound of every device wait and the test hook that withholds barrier
 * arrivals are read from the environment at each call, as rteaal_sim_create
 * reads them (RTEAAL_BARRIER_TIMEOUT_NS, RTEAAL_TEST_WITHHOLD_ARRIVAL).
 * cycles: host [n_lanes] per-lane cycle counts, or NULL to run uniform_cycles.
 * stim_mode: RTEAAL_STIM_HOLD or RTEAAL_STIM_XORSHIFT.  flags: RTEAAL_STEP_RESET.
 * Sizes beyond RTEAAL_STATIC_MAX_LANES lanes are rejected (E_INVALID).
 * The first call on each device looks up the array's device address (make it
 * before any stream capture).  Every call shares the one array and leaves its
 * contents behind; the barrier and error words are cleared at the start of
 * each call.  Calls that overlap on the GPU (other streams, other threads) race
 * on the array: serialise them.  Synchronises stream; returns E_TIMEOUT if a
 * bounded barrier wait gave up. */
#define RTEAAL_STATIC_MAX_LANES 65536u
int rteaal_step_static(const rteaal_design *design, void *state, uint64_t *mem, uint64_t *xs,
                       uint32_t n_lanes, const uint32_t *cycles, uint32_t uniform_cycles,
                       int stim_mode, uint32_t flags, void *stream);

/* Thread-local description of the last failure on this thread. */
const char *rteaal_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RTEAAL_H */
