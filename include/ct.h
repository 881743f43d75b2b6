/*
 * ct.h -- C ABI of the GB300 Compact-Table propagation library (libct.so).
 *
 * The library propagates table constraints with the Compact-Table (CT)
 * algorithm of "GPU Accelerated Compact-Table Propagation" (Santi, Tardivo,
 * Dovier, Formisano, 2025): Algorithm 1 (enforceGAC), Algorithm 2
 * (updateTable, with both the delta and the reset mask) and Algorithm 3
 * (filterDomains, with residues), run as CUDA kernels on one GPU with all
 * table state resident in device memory. A table constraint, its currTable
 * and its supports bitsets are defined in Sec. 2 (Table 1); the serial data
 * structures (_supports, _supportJmp, _variablesOffsets, 32-bit words) in
 * Sec. 3; the GPU propagators that this design generalises in Sec. 4.
 *
 * Conventions shared by every call
 * --------------------------------
 * Return value: CT_OK (0), CT_INFEASIBLE (1, the constraint or the network has
 *   no solution under the given domains -- a CSP failure in the sense of
 *   Algorithm 1, not an error) or a negative CT_ERR_* code. After an error,
 *   ct_last_error() returns a message for the calling thread.
 * Domains: the domain of a variable with initial range
 *   [dom_lo, dom_lo + dom_size) is a bitset of ceil(dom_size / 32) uint32
 *   words; value v is bit (v - dom_lo) % 32 of word (v - dom_lo) / 32 (least
 *   significant bit first). Bits at or above dom_size must be zero. The
 *   domains of a table's scope are stored back to back in scope order.
 * Words: currTable and the supports rows are 32-bit words (Sec. 3), tuple j
 *   at bit j % 32 of word j / 32, where j counts the retained tuples (tuples
 *   with every value inside the initial domains, in input order; duplicates
 *   are kept).
 * Ownership: the caller owns every buffer it passes; the library copies what
 *   it keeps (tuples, scopes, domains) during the call. Handles belong to the
 *   caller until the matching destroy call.
 * Streams and threads: every handle runs its work on one CUDA stream (the
 *   stream given at creation, or a stream the library creates). A handle must
 *   not be used from two host threads at once; distinct handles may.
 * Device pointers: arguments documented as "device" must point to memory of
 *   the current CUDA device that the handle's stream can access.
 */
#ifndef CT_H
#define CT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CT_OK 0
#define CT_INFEASIBLE 1
#define CT_ERR_ARG (-1)     /* invalid argument (null pointer, bad size, duplicate scope variable) */
#define CT_ERR_OOM (-2)     /* host or device allocation failed */
#define CT_ERR_CUDA (-3)    /* a CUDA call failed; see ct_last_error() */
#define CT_ERR_STATE (-4)   /* domains grew without a restore, or use after a failure without restore */
#define CT_ERR_TIMEOUT (-5) /* a bounded device-side wait ran out */
#define CT_ERR_LEVEL (-6)   /* restore to a level that is not on the stack */

typedef struct ct_table ct_table;
typedef struct ct_model ct_model;

/* Tuning knobs; a zeroed struct (or NULL) selects the defaults. */
typedef struct ct_options {
    int32_t reserved0;        /* must be 0 */
    int32_t grid_blocks;      /* 0 = auto; CTAs of the cooperative propagation launch (capped at residency) */
    int32_t no_residues;      /* 1 = skip the residue probe and scan for every value */
    int32_t profile;          /* 1 = time each kernel with CUDA events (see ct_get_profile) */
    int32_t host_fixpoint;    /* models: 1 = run the fixpoint queue on the host, one launch per table
                                 propagation (default: the whole fixpoint in one launch) */
    int32_t autotune;         /* 1 = pick the launch shape at creation by timing trial propagations:
                                 for a table, batches of 16 or 8 row loads in flight (2 or 3 CTAs
                                 per SM) and the CTA count (segments per CTA); for a model, the CTA
                                 count of the fixpoint launch (tables and segments per CTA). The
                                 trials run between a save and a restore, so the state is unchanged.
                                 Ignored when grid_blocks is set. */
    int32_t copy_state;       /* 1 = ablation of the paper's propagators (Sec. 4: CT_CU^u/^f/^uf copy
                                 _currTable host->device before and device->host after every
                                 propagation): ct_propagate round-trips currTable through a pinned
                                 host copy each call (and ct_restore refreshes it). Results are the
                                 same; only the copies' cost is added. */
    int32_t shard;            /* 1 = the table is one word-range shard of a larger table (the
                                 data-parallel split of one table, see ct_sharded_create):
                                 filterDomains clears the values none of THIS table's valid
                                 tuples supports, an empty currTable is not a failure (every
                                 value is cleared, status CT_OK), and the last-seen domains keep
                                 the call's input domains, since another shard may support a
                                 value this one cleared. Positive tables only. */
    int32_t no_split;         /* 1 = updateTable gives each 32-chunk segment to one warp, which walks
                                 the call's whole row list (default: the row list of a segment is
                                 cut over up to 8 warps of a CTA, one batch of row loads each where
                                 the list allows, and their partial masks are combined in shared
                                 memory; results are the same). */
    int32_t no_early_filter;  /* 1 = filterDomains always waits for the whole update (a grid barrier).
                                 Default: a call that ORs at most 16 supports rows (8 on tables of more
                                 segments than one wave of warps) while at least half the currTable
                                 chunks are live filters beside the update, each probed chunk
                                 recomputed from its stored value and the call's rows (Algorithm 2 at
                                 one chunk), and one grid barrier ends both; positive tables with
                                 residues and a plan in shared memory. Results are the same. */
} ct_options;

/* Static shape and live state of a table (ct_get_info). */
typedef struct ct_table_info {
    int32_t arity;
    int32_t rows;          /* supports rows = sum of the initial domain sizes (_supportSize, Sec. 3) */
    int64_t tuples;        /* retained tuples t */
    int64_t words;         /* ceil(t / 32) 32-bit currTable words (_currTableSize, Sec. 3) */
    int64_t chunks;        /* ceil(words / 4): 128-bit units of the sparse index */
    int32_t segments;      /* segments of 32 chunks; the non-zero index keeps one live mask per segment */
    int32_t seg_capacity;  /* chunks per segment (32) */
    int64_t live_chunks;   /* chunks currently in the non-zero index */
    int64_t trail_size;    /* trail entries in use */
    int32_t depth;         /* saved levels on the stack */
    int32_t local_plan;    /* 1: every CTA computes the update plan in shared memory */
    int32_t grid_blocks;   /* CTAs of the propagation launch */
    int32_t short_tuples;  /* retained tuples with at least one CT_STAR component */
    int64_t device_bytes;  /* device memory held by the table */
    int32_t loads_in_flight; /* 16 (2 CTAs per SM) or 8 (3 CTAs per SM) row loads per lane */
    int32_t autotuned;     /* 1 if the launch shape was chosen by trial propagations */
} ct_table_info;

/* Figures of the last ct_propagate call (ct_get_call_stats). */
typedef struct ct_call_stats {
    int32_t status;
    int32_t changed_vars;   /* |s_val|: scope variables whose domain shrank since the last call */
    int32_t delta_vars;     /* of those, masked with the removed values (|Delta| < |dom|) */
    int32_t reset_vars;     /* of those, masked with the remaining values */
    int32_t rows_ored;      /* supports rows OR-ed by updateTable (sum of k_i) */
    int32_t sup_vars;       /* |s_sup|: scope variables with more than one value */
    int32_t residue_hits;   /* values found supported by their residue chunk */
    int32_t local_found;    /* values found in the 32-chunk windows after a missed residue */
    int32_t hard;           /* values that needed the full index scan */
    int32_t windows;        /* 32-chunk windows probed */
    int32_t pruned;         /* values removed by filterDomains */
    int32_t trail_added;    /* trail entries appended */
    int64_t live_chunks_in;  /* non-zero index size at entry (128-bit chunks) */
    int64_t live_chunks_out; /* ... and at exit */
    int64_t live_words_in;   /* non-zero 32-bit currTable words at entry (N) */
    int64_t update_bytes;    /* algorithmic bytes of updateTable: 4 * N * (rows_ored + 2), 0 if no row */
    int64_t filter_bytes;    /* algorithmic bytes of filterDomains: 4 * supports words tested */
    int32_t phase_ns[4];     /* %globaltimer, ns from the first CTA's start to: plan done, update done,
                                probes done, result published (device-side, no launch latency) */
    int32_t early_filter;    /* 1: filterDomains ran beside updateTable (ct_options.no_early_filter) */
} ct_call_stats;

/* Accumulated launch times (ct_options.profile = 1): CUDA events recorded on
 * the table's stream right before and after each propagation launch. */
typedef struct ct_profile {
    int64_t calls;
    double kernel_ms;     /* sum of the event intervals around the propagation kernel */
    int64_t update_bytes; /* sum of ct_call_stats.update_bytes */
    int64_t filter_bytes; /* sum of ct_call_stats.filter_bytes */
    double device_ms;     /* sum of ct_call_stats.phase_ns[3] (kernel time without launch latency) */
    double host_ms;       /* wall time spent inside the propagation calls */
    double launch_ms;     /* ... of which in the launch call */
    double wait_ms;       /* ... of which waiting for the result */
} ct_profile;

/* The wildcard component of a short tuple (any value of the variable). */
#define CT_STAR ((int32_t)(-2147483647 - 1))

/* ---------------------------------------------------------------- table --
 * ct_create: build a table constraint (Sec. 2; constructor of class Table,
 * Sec. 3, and its device copy, Sec. 4).
 *   arity      number of scope variables (1 .. 2048)
 *   dom_lo     host int32[arity]: first value of each initial domain
 *              (_variablesOffsets, Sec. 3)
 *   dom_size   host int32[arity]: initial domain sizes (1 .. 65536)
 *   tuples     host int32[t * arity], row-major: tuple j is
 *              tuples[j*arity .. j*arity+arity-1]; may be NULL when t == 0
 *   t          number of input tuples (>= 0)
 *   opt        tuning knobs or NULL
 *   cuda_stream cudaStream_t to run on, or NULL for a stream owned by the table
 *   out        receives the handle (also on CT_INFEASIBLE)
 * A component equal to CT_STAR is a wildcard ("*", any value of the
 * variable): short tables, the extension of Compact-Table to short tuples
 * that the paper cites (Sec. 1) but does not evaluate. A short tuple stands
 * for every tuple obtained by replacing its wildcards with values; it is
 * valid while its other components are in their domains. Its supports rows
 * hold it for every value of a wildcard position (filtering and the reset
 * update); the delta update removes only tuples whose component equals a
 * removed value.
 * Tuples with a value outside the initial domains are dropped. Returns
 * CT_INFEASIBLE when no tuple is left (the constructor's unsatisfiability
 * check, Sec. 3); the handle is still valid and every propagation of it
 * fails. The first ct_propagate starts from the initial domains, so values
 * already removed by the caller count as removed since the last call.
 */
/* ct_create_negative: a negative table (the tuples are the FORBIDDEN ones), the
 * extension of Compact-Table to negative tables that the paper cites (Sec. 1)
 * but does not evaluate. Arguments as ct_create; duplicate tuples count once,
 * wildcards are refused. currTable holds the valid forbidden tuples; value a
 * of scope variable x keeps its support while the valid forbidden tuples with
 * x = a are fewer than prod_{y != x} |D(y)| (popcount of supports[x,a] AND
 * currTable, counted only when that product does not exceed the valid
 * forbidden tuples). A negative table never fails because its currTable is
 * empty. One ct_propagate is one such filtering pass over the input domains;
 * unlike a positive table's it is not always a fixpoint (a removal shrinks
 * the other variables' products): call again until nothing changes (a model
 * does so). Limits: arity <= 512, <= 2,048 domain words, <= 4,096 values;
 * CT_ERR_ARG when no tuple is inside the domains. */
int ct_create_negative(int arity, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples,
                       int64_t t, const ct_options* opt, void* cuda_stream, ct_table** out);

int ct_create(int arity, const int32_t* dom_lo, const int32_t* dom_size,
              const int32_t* tuples, int64_t t, const ct_options* opt,
              void* cuda_stream, ct_table** out);

/* ct_propagate: enforce GAC on the table (Algorithm 1: change detection,
 * updateTable of Algorithm 2, failure test, filterDomains of Algorithm 3).
 *   dom_bits      device uint32, in/out: the scope domains (layout above).
 *                 They must be subsets of the domains at the end of the
 *                 previous call (or at the restored level); otherwise
 *                 CT_ERR_STATE. On CT_OK the unsupported values are cleared.
 *   changed_vars  host uint32[ceil(arity/32)] or NULL: bit i set iff the call
 *                 removed a value of scope variable i.
 * Blocks until the result is known (one small device-to-host copy). On
 * CT_INFEASIBLE the domain contents are unspecified and the table must be
 * restored (ct_restore) before it is propagated again.
 */
int ct_propagate(ct_table* ct, uint32_t* dom_bits, uint32_t* changed_vars);

/* ct_propagate_host: as ct_propagate, with dom_bits in host memory, filtered
 * in place on CT_OK. Domains of at most 16 words in all (tables whose plan
 * fits in shared memory) travel to the device inside the launch's parameters,
 * larger ones by a copy; the filtered domains come back through the mapped
 * status block of the call. */
int ct_propagate_host(ct_table* ct, uint32_t* dom_bits_host, uint32_t* changed_vars);

/* ct_save: push a backtrack level (the trail of Sec. 4: MiniCP alternates
 * search and propagation with backtracking). *level_out receives the level
 * number (the stack depth before the push, starting at 0). */
int ct_save(ct_table* ct, int* level_out);

/* ct_restore: return currTable, its non-zero index and the last-seen domains
 * to their state at ct_save(level), and drop that level and every level
 * above it (depth becomes `level`). CT_ERR_LEVEL if level is not in
 * [0, depth). Residues are hints and are not restored. */
int ct_restore(ct_table* ct, int level);

/* ct_get_currtable: copy currTable (Sec. 2, Table 1(c)) to the host.
 *   words_host          host uint32[ceil(t/32)] or NULL
 *   nonzero_words_out   host or NULL: number of non-zero 32-bit words */
int ct_get_currtable(ct_table* ct, uint32_t* words_host, int64_t* nonzero_words_out);

/* ct_get_support_row: copy supports row `row` (Sec. 2, Table 1(b); row of
 * value v of scope variable i = sum of the first i domain sizes + v - dom_lo[i],
 * _supportJmp of Sec. 3) to host uint32[ceil(t/32)]. */
int ct_get_support_row(ct_table* ct, int row, uint32_t* words_host);

/* ct_get_index: copy the non-zero index (128-bit chunk numbers, each live
 * chunk exactly once, ascending) to host int32[live_chunks]; *count_out
 * receives live_chunks. index_host may be NULL. */
int ct_get_index(ct_table* ct, int32_t* index_host, int64_t* count_out);

int ct_get_info(ct_table* ct, ct_table_info* info);
int ct_get_call_stats(ct_table* ct, ct_call_stats* stats);
int ct_get_profile(ct_table* ct, ct_profile* prof);
int ct_reset_profile(ct_table* ct);
/* ct_set_profile: switch the per-launch timing of ct_options.profile on (1)
 * or off (0) for the following calls; accumulated figures are kept (pending
 * timings are collected before switching off). */
int ct_set_profile(ct_table* ct, int on);

/* ct_destroy: free the table (NULL is accepted). */
int ct_destroy(ct_table* ct);

/* ct_arm_wait_timeout: test hook for the bounded device waits (no fault, no
 * hang). The next ct_propagate on `ct` (ct == NULL: the next
 * ct_propagate_noalloc on the calling thread's current device) starts with its
 * grid barrier's arrival count set where no CTA can complete it, and with each
 * barrier wait limited to `polls` polls (> 0): every wait runs out, the kernel
 * records CT_ERR_TIMEOUT and returns without publishing, and that call
 * returns CT_ERR_TIMEOUT. A table whose wait ran out refuses every later
 * propagate and restore with CT_ERR_TIMEOUT (destroy it); the allocation-free
 * entry point starts afresh on its next call. Returns CT_ERR_ARG for polls == 0. */
int ct_arm_wait_timeout(ct_table* ct, uint32_t polls);

/* ct_propagate_noalloc: one propagation of a table held entirely in buffers
 * the caller owns, for callers that cannot allocate device memory when they
 * propagate (a framework's memory pool owns the device, allocation is only
 * allowed at start-up, or the implicit synchronisation of cudaMalloc/cudaFree
 * is not acceptable). The paper has no counterpart; it is a convenience of this
 * library. Same computation as ct_propagate (change detection, updateTable,
 * failure test, filterDomains), without backtrack levels.
 *   arity         1 .. 16 scope variables
 *   dom_size      host int32[arity]; the sum of the sizes (supports rows) at most 1024
 *   t             tuples, 1 .. 8,388,608
 *   supports      device, 16-byte aligned: sum(dom_size) rows of Wp = 4*ceil(ceil(t/32)/4)
 *                 uint32 words; row sum(dom_size[0..i-1]) + a holds bit j for every
 *                 tuple j whose i-th value is dom_lo[i] + a (ct_get_support_row gives them)
 *   curr_table    device, 16-byte aligned, in/out: Wp words of currTable; first call:
 *                 the bits of the t tuples set, later calls: the previous output
 *   dom_bits      device, in/out: the scope domains (layout above); filtered on CT_OK
 *   last_dom_bits device, in/out: the domains at the end of the previous call (the full
 *                 initial domains for the first call); dom_bits must be a subset
 *   changed_vars  host uint32[1] or NULL: bit i set iff the call removed a value of x_i
 *   cuda_stream   stream to run on (NULL: the legacy default stream); the call blocks
 *                 until the result is known
 * It allocates nothing: its scratch is one static device array of about 32 KB
 * that every GPU loading the library keeps until the process exits. The first
 * call on a device looks the array's device address up (and the kernel's
 * residency). All calls on a
 * device share the array and it keeps the last call's contents (each call
 * clears what it needs cleared), so calls that overlap on the GPU -- two host
 * threads, or two streams -- race and must be serialised by the caller.
 * Sizes beyond the limits return CT_ERR_ARG with a message. */
int ct_propagate_noalloc(int arity, const int32_t* dom_size, int64_t t, const uint32_t* supports,
                         uint32_t* curr_table, uint32_t* dom_bits, uint32_t* last_dom_bits,
                         uint32_t* changed_vars, void* cuda_stream);

/* ------------------------------------------------------ word-range shards --
 * One table split into K shards of contiguous retained tuples (whole 128-tuple
 * chunks of currTable), run on one device: the data-parallel split of one
 * table's propagation. updateTable is local to each shard; a value is
 * supported iff some valid tuple of some shard carries it (the GAC definition
 * of Sec. 2), so the domains are the OR of what each shard supports, and the
 * table fails iff every shard's currTable is empty. The OR runs as one small
 * kernel here, where a split over several GPUs would all-reduce the bits.
 */
typedef struct ct_sharded ct_sharded;

/* ct_shard_bounds: the split of t >= 1 retained tuples into K shards of whole
 * 128-tuple chunks (host only): bounds_out (host int64[K + 1]) receives
 * bounds_out[0] = 0 < bounds_out[1] < ... < bounds_out[K] = t, shard k holding
 * tuples [bounds_out[k], bounds_out[k + 1]), each bound but the last a
 * multiple of 128 and every shard non-empty. CT_ERR_ARG if K > ceil(t / 128). */
int ct_shard_bounds(int64_t t, int K, int64_t* bounds_out);

/* ct_sharded_create: the table of ct_create (same arguments and conventions;
 * positive tables, wildcards allowed) split by ct_shard_bounds over its
 * retained tuples into K tables created with ct_options.shard = 1 on one
 * stream. CT_INFEASIBLE and no handle when no tuple is inside the domains. */
int ct_sharded_create(int arity, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples,
                      int64_t t, int K, const ct_options* opt, void* cuda_stream, ct_sharded** out);

/* ct_sharded_propagate: ct_propagate of the whole table. Every shard filters
 * its own device copy of dom_bits, and dom_bits (device, in/out) becomes the
 * OR of the copies. changed_vars as in ct_propagate. CT_INFEASIBLE iff a
 * domain became empty; the shards are then restored with ct_sharded_restore
 * before the next call. dom_bits is read and written on the stream given to
 * ct_sharded_create; the call blocks until the result is known. */
int ct_sharded_propagate(ct_sharded* sh, uint32_t* dom_bits, uint32_t* changed_vars);

/* ct_sharded_save / ct_sharded_restore: ct_save / ct_restore on every shard
 * (the shards' level stacks stay equal). */
int ct_sharded_save(ct_sharded* sh, int* level_out);
int ct_sharded_restore(ct_sharded* sh, int level);

/* ct_sharded_get_currtable: currTable of the whole table (host
 * uint32[ceil(t/32)] or NULL, t the retained tuples): shard k's words at word
 * bounds[k] / 32; *nonzero_words_out (or NULL) the non-zero words of all. */
int ct_sharded_get_currtable(ct_sharded* sh, uint32_t* words_host, int64_t* nonzero_words_out);

/* ct_sharded_get_shard: shard k's table handle, owned by sh (for its
 * statistics and info; propagate it only through ct_sharded_propagate). */
int ct_sharded_get_shard(ct_sharded* sh, int k, ct_table** table_out);

/* ct_sharded_destroy: free the shards (NULL is accepted). */
int ct_sharded_destroy(ct_sharded* sh);

/* ---------------------------------------------------------------- model --
 * A model is a set of integer variables and table constraints over them,
 * propagated to a common fixpoint (Sec. 2: propagation removes unsupported
 * values until GAC holds everywhere or a failure is found) and searched
 * depth-first (Sec. 4). Domains of all variables live on the device in the
 * layout above, variable after variable.
 */
typedef struct ct_search_stats {
    int64_t nodes;        /* fixpoints computed on search nodes, root and failed nodes included */
    int64_t fails;        /* nodes whose fixpoint failed */
    int64_t solutions;    /* nodes where every variable is fixed after propagation */
    int64_t propagations; /* table propagations (ct_propagate-equivalent calls) */
    int32_t max_depth;
    int32_t complete;     /* 1 if the tree was exhausted or the first solution found as asked */
    double seconds;
} ct_search_stats;

/* ct_model_create: nvars variables with initial ranges [dom_lo[v], dom_lo[v] + dom_size[v]). */
int ct_model_create(int nvars, const int32_t* dom_lo, const int32_t* dom_size,
                    const ct_options* opt, void* cuda_stream, ct_model** out);

/* ct_model_add_table: add a table over `scope` (host int32[arity] of distinct
 * variable indices); tuples as in ct_create. CT_INFEASIBLE if no tuple fits
 * the initial domains (the model then has no solution). */
int ct_model_add_table(ct_model* m, const int32_t* scope, int arity,
                       const int32_t* tuples, int64_t t);

/* ct_model_add_negative_table: a negative table (see ct_create_negative) over
 * `scope`. The one-launch fixpoint kernel and the batched searches propagate
 * it beside the positive tables: a value whose valid forbidden tuples number
 * as many as the combinations of the other scope domains is removed, and the
 * table runs again after its own removals (one pass of a negative table is
 * not GAC for it). A model holding one refuses features and lookahead
 * (CT_ERR_ARG). */
int ct_model_add_negative_table(ct_model* m, const int32_t* scope, int arity, const int32_t* tuples, int64_t t);

/* ct_model_propagate: run table propagations until no domain changes
 * (fixpoint) or a table fails (CT_INFEASIBLE). */
int ct_model_propagate(ct_model* m);

/* ct_model_get_domains / ct_model_set_domains: host copies of all domains
 * (sum over variables of ceil(dom_size/32) words). Set domains must be
 * subsets of the current ones. */
int ct_model_get_domains(ct_model* m, uint32_t* words_host);
int ct_model_set_domains(ct_model* m, const uint32_t* words_host);

/* Counters of the model's fixpoints since creation or ct_model_reset_stats
 * (the one-launch fixpoint fills all of them; the host queue only
 * propagations). Bytes are algorithmic, as for one table: updateTable
 * 4 * (non-zero words at entry) * (rows OR-ed + 2) per table propagation;
 * filterDomains 16 per residue hit, 512 per window probed and 16 per live
 * chunk of every full scan. */
typedef struct ct_model_stats {
    int64_t fixpoints;     /* launches of the fixpoint kernel */
    int64_t rounds;        /* Jacobi rounds in them */
    int64_t propagations;  /* table propagations */
    int64_t residue_hits;
    int64_t window_hits;
    int64_t hard_values;
    int64_t update_bytes;
    int64_t filter_bytes;
    double wait_seconds;   /* host time from each launch to its published result */
    double phase_seconds[8]; /* with ct_options.profile: fixpoint kernel time by phase, as in
                                ct_batch_info (prologue, plan, updateTable, residue probes,
                                index scans, removals, next-round selection, publication) */
} ct_model_stats;
int ct_model_get_stats(ct_model* m, ct_model_stats* out);
int ct_model_reset_stats(ct_model* m);

int ct_model_save(ct_model* m, int* level_out);
int ct_model_restore(ct_model* m, int level);

/* ct_search_dfs: depth-first search with first-fail binary branching: the
 * unfixed variable with the smallest domain (ties: lowest index); left branch
 * x = min(dom x), right branch x != min(dom x). Propagates at every node.
 *   node_limit      stop after this many nodes (<= 0: no limit)
 *   count_all       0: stop at the first solution; 1: count all solutions
 *   out             host, receives the counters
 *   first_solution  host int32[nvars] or NULL: values of the first solution
 * Returns CT_OK whether or not a solution exists; the model's domains are
 * back at their state before the call. */
int ct_search_dfs(ct_model* m, int64_t node_limit, int count_all,
                  ct_search_stats* out, int32_t* first_solution);

/* ct_search_batch: the search of ct_search_dfs (same branching, same counts
 * when count_all = 1 and node_limit <= 0) with many search nodes propagated
 * together. Not in the paper, whose solver propagates one node at a time
 * (Sec. 4); this is the batched driver of the search. The tree is first
 * expanded depth-first down to split_depth on the model itself; the nodes
 * found there ("open nodes", kept in depth-first order) are handed to `slots`
 * copies of the network (the copies share the supports rows of the model's
 * tables and own their currTable, index, trail and levels). Every slot
 * searches the subtree of one open node depth-first; one cooperative launch
 * per step undoes the trails the slots backtrack over and propagates the
 * current node of every active slot to its fixpoint. A slot whose subtree is
 * done takes the next open node, or else the untried right branch nearest the
 * root of another slot's subtree.
 *   slots        1 .. 4096 copies; slots x tables <= 1,048,576
 *   split_depth  0 .. 64 (0: the root itself is the only open node)
 *   node_limit   stop issuing nodes after this many (<= 0: no limit); the
 *                nodes visited then differ from ct_search_dfs's
 *   count_all    1: count every solution; 0: stop once the first solution in
 *                depth-first order is known (nodes after it are not started,
 *                nodes before it are finished), so first_solution equals
 *                ct_search_dfs's while nodes and fails can differ; 2: stop at
 *                the first solution any slot finds (no new node is started;
 *                the nodes of that launch still finish); in this mode the
 *                model first searches depth-first alone for up to 4 nodes per
 *                slot (above split_depth), and the open nodes are the nodes
 *                at split_depth plus the frontier that search leaves (the node
 *                it stopped at and every untried right branch above it)
 *   out          host, receives the counters as in ct_search_dfs
 *   first_solution  host int32[nvars] or NULL: the first solution in
 *                depth-first order among those found (with count_all = 1, or
 *                with count_all = 0 and no node limit, ct_search_dfs's)
 * Returns CT_ERR_ARG for count_all outside 0..2.
 *   info         host or NULL: counters of the batching itself
 * Returns CT_OK, CT_ERR_ARG (bad sizes), CT_ERR_STATE (a failed model),
 * CT_ERR_OOM, CT_ERR_CUDA or CT_ERR_TIMEOUT. The model's domains and tables
 * are back at their state before the call; the copies are kept for the next
 * call with the same number of slots and freed by ct_model_destroy. */
typedef struct ct_batch_info {
    int64_t open_nodes;   /* nodes handed to the slots at split_depth */
    int64_t split_nodes;  /* nodes propagated on the model itself above split_depth */
    int64_t steps;        /* cooperative launches of the slots' phase */
    int64_t steals;       /* right branches taken over from another slot */
    int64_t slot_nodes;   /* node propagations done in the slots */
    int64_t rounds;       /* fixpoint rounds summed over the launches */
    int64_t residue_hits; /* slots' phase, Algorithm 3: values whose residue still held a support, */
    int64_t window_hits;  /* values found in the windows after the residue, */
    int64_t hard_values;  /* values left for the full index scan (found or pruned there) */
    int64_t update_bytes; /* slots' phase: algorithmic bytes as in ct_model_stats */
    int64_t filter_bytes;
    int32_t slots;
    int32_t split_depth;
    double setup_seconds; /* building or refreshing the copies */
    double wait_seconds;  /* slots' phase: from each launch to its results on the host */
    double slot_seconds;  /* slots' phase in all (host work, copies, launches and waits) */
    double phase_seconds[8]; /* with ct_options.profile: fixpoint kernel time by phase (prologue,
                                plan, updateTable, residue probes, index scans, removals,
                                next-round selection, publication) */
} ct_batch_info;

int ct_search_batch(ct_model* m, int slots, int split_depth, int64_t node_limit, int count_all,
                    ct_search_stats* out, int32_t* first_solution, ct_batch_info* info);

/* ct_search_batch_assign: ct_search_batch with the tree split where a node's
 * path holds `assign_depth` assignments (left branches x = v) instead of at a
 * number of binary levels: every node above the split is expanded breadth-first
 * in the slots (a right branch x != v keeps its parent's count), and the nodes
 * that reach assign_depth assignments are the open nodes, put in depth-first
 * order. The tree is the one ct_search_dfs visits, so with count_all = 1 and
 * no node limit the counts equal its counts. This reads "search nodes split
 * at depth d" of a d-way enumeration as d assignments of the binary tree.
 *   assign_depth 1 .. 16; count_all 0 or 1 (else CT_ERR_ARG); the rest as in
 *                ct_search_batch (info->open_nodes: the open nodes made). */
int ct_search_batch_assign(ct_model* m, int slots, int assign_depth, int64_t node_limit, int count_all,
                           ct_search_stats* out, int32_t* first_solution, ct_batch_info* info);

/* ct_search_batch_device: ct_search_batch counting every solution (count_all
 * = 1, first-fail branching, no policy) with the slots' search run on the
 * device instead of stepped by the host. The tree above split_depth is
 * expanded as by ct_search_batch; its open nodes go to a device queue, and
 * the fixpoint kernel, between its rounds, moves every slot whose node is at
 * its fixpoint (or failed) on: branch on the first-fail variable, backtrack
 * to the deepest untried right branch (trails undone and index snapshots
 * restored on the device), or take the next open node. Each launch runs at
 * most 1,024 rounds; the host launches again until every slot is idle and
 * the queue is empty. The device keeps, per slot, up to L levels below its
 * open node and, per table copy, a trail of F x its chunks + 1,024 entries;
 * a deeper subtree or a fuller trail makes the host rebuild them with L or F
 * doubled and run the device search again (L from 64 to 1,024, F from 16 to
 * 128; beyond those CT_ERR_LEVEL or CT_ERR_OOM). With no node limit the
 * counts and the first solution equal ct_search_dfs's. Slots do not take
 * right branches from each other here: the breadth-first split goes on below
 * split_depth until there are at least two open nodes per slot (or depth 48).
 *   slots 1 .. 4096, split_depth 0 .. 64, node_limit as in ct_search_batch;
 *   CT_ERR_ARG when the model has a policy (ct_model_set_policy). */
int ct_search_batch_device(ct_model* m, int slots, int split_depth, int64_t node_limit, ct_search_stats* out,
                           int32_t* first_solution, ct_batch_info* info);

int ct_model_destroy(ct_model* m);

/* ------------------------------------------------------- learned order -- */
/* Not in the paper, whose solver branches first-fail (Sec. 4): a small network
 * scores the unfixed variables of a search node and the search branches on
 * the best one (ties to the lowest index); values stay min-first, so every
 * propagated domain is the same GAC fixpoint as with first-fail.
 *
 * Features of variable x (8 floats; all 0 when |D(x)| < 2). s = |D(x)|, d0 its
 * initial size, deg(x) the tables holding x (degmax the largest, >= 1), smax
 * the largest |D| among unfixed variables; for every table c holding x with
 * live_c > 0 valid tuples (the set bits of its currTable),
 * p_c(a) = popcount(supports[x,a] AND currTable_c) / live_c for a in D(x):
 *   f0 = s/d0, f1 = log2(s)/8, f2 = deg/degmax, f3 = mean_c s*min_a p_c(a),
 *   f4 = mean_c max_a p_c(a), f5 = mean_c (-sum_a p_c(a) log2 p_c(a))/log2(s),
 *   f6 = mean_c log2(1 + live_c)/32, f7 = s/smax
 * (f3-f6 are 0 when no table holding x has a valid tuple).
 *
 * Network: float32, 8 -> 64 -> 64 -> 1, ReLU after the first two layers;
 * CT_MLP_WEIGHTS floats, flat: W1[64][8], b1[64], W2[64][64], b2[64], W3[64],
 * b3 (rows are output units). Training minimises sum (out - y)^2 / (2B) per
 * batch of B samples with Adam (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected); its state persists across ct_mlp_train calls and is reset
 * by ct_mlp_set_weights. */
#define CT_MLP_FEATURES 8
#define CT_MLP_HIDDEN 64
#define CT_MLP_WEIGHTS 4801
#define CT_MLP_MAX_BATCH 128

typedef struct ct_mlp ct_mlp;

/* ct_mlp_create: a network with the given weights (host, CT_MLP_WEIGHTS
 * floats, copied) on `cuda_stream` (NULL: a library-created stream). */
int ct_mlp_create(const float* weights_host, void* cuda_stream, ct_mlp** out);
int ct_mlp_set_weights(ct_mlp* m, const float* weights_host);
int ct_mlp_get_weights(ct_mlp* m, float* weights_host);
/* ct_mlp_forward: scores of n feature rows; x_dev float[n][8] and scores_dev
 * float[n] are device buffers of the caller; stream-ordered, no sync. */
int ct_mlp_forward(ct_mlp* m, const float* x_dev, int64_t n, float* scores_dev);
/* ct_mlp_grad: loss and gradient (host float[CT_MLP_WEIGHTS]) of one batch of
 * 1 <= n <= CT_MLP_MAX_BATCH host rows; the weights do not change. */
int ct_mlp_grad(ct_mlp* m, const float* x_host, const float* y_host, int n, float* loss_out, float* grad_host);
/* ct_mlp_train: Adam over `epochs` passes; pass e visits the samples in the
 * order orders_host[e*n .. e*n+n) (a permutation of 0..n-1 per epoch) in
 * consecutive batches of `batch` <= CT_MLP_MAX_BATCH (the last may be
 * shorter). epoch_loss_host (float[epochs] or NULL) receives each epoch's mean
 * batch loss. One kernel launch; inputs are copied to the device. */
int ct_mlp_train(ct_mlp* m, const float* x_host, const float* y_host, int64_t n, const int32_t* orders_host,
                 int epochs, int batch, float lr, float* epoch_loss_host);
int ct_mlp_destroy(ct_mlp* m);

/* ct_model_features: features (host float[nvars][8]) of the model's current
 * state (after ct_model_propagate; CT_ERR_STATE on a failed model). */
int ct_model_features(ct_model* m, float* features_host);
/* ct_model_set_policy: branch with the network's scores in ct_search_dfs and
 * ct_search_batch (NULL: first-fail). The network must outlive its use. */
int ct_model_set_policy(ct_model* m, ct_mlp* policy);
/* ct_model_set_trace: ct_search_dfs records the branching variable of every
 * branching node, in depth-first order, into decisions_host[0 .. capacity)
 * and the number recorded into *count_host (NULL buffer: no trace). */
int ct_model_set_trace(ct_model* m, int32_t* decisions_host, int64_t capacity, int64_t* count_host);
/* ct_model_lookahead: labels (host float[nvars]) of the model's state after
 * ct_model_propagate: for each unfixed variable x, the fixpoint of D with
 * D(x) := {min D(x)} is computed on the slot copies of the batched search
 * (`slots` at a time); label 1 if it fails, else (L - L')/L with
 * L = sum_v log2|D_v| before and L' after. NaN for fixed variables. */
int ct_model_lookahead(ct_model* m, int slots, float* labels_host);
/* ct_search_collect: the first-fail search of ct_search_dfs (any policy set is
 * ignored) for at most node_limit nodes; at every branching node the features
 * and lookahead labels of its unfixed variables are appended as samples
 * (features_host float[max_samples][8], labels_host float[max_samples]) until
 * max_samples. *samples_out receives the count. The model is back at its
 * state before the call. */
int ct_search_collect(ct_model* m, int64_t node_limit, int slots, int64_t max_samples, float* features_host,
                      float* labels_host, int64_t* samples_out);

/* ------------------------------------------------------------ test hooks -- */
/* For tests of the library itself (no counterpart in the paper), off by
 * default; they cover the device buffers a table owns: those ct_create
 * allocates, the trail and the level stack (not the buffers of models and
 * batched searches, nor arenas of table copies). Process-wide settings; each
 * returns CT_OK unless stated.
 *
 * ct_debug_guard_buffers: while on (1), tables created afterwards put 256
 * bytes of guard before and after every such buffer, filled with 0xA5 (the
 * buffers keep their 256-byte alignment); 0 switches it off for later tables.
 * No kernel addresses a guard, so a changed guard byte means a write outside
 * a buffer (compute-sanitizer being unavailable where this library runs).
 *
 * ct_debug_check_guards: waits for the device and writes to *changed_out how
 * many guard bytes of ct's buffers differ from 0xA5 (0 for a table created
 * without guards). poke > 0 first overwrites `poke` bytes of the first
 * buffer's leading guard with zeros, by a host-side memset (a check of the
 * check itself); 0 <= poke <= 256, else CT_ERR_ARG.
 *
 * ct_debug_fail_alloc: after n more device allocations of table buffers the
 * next one fails as if the device were out of memory (the call that made it
 * returns CT_ERR_OOM and releases what it took); one failure per arming;
 * n < 0 disarms.
 *
 * ct_debug_device_bytes: bytes of device memory the table buffers hold now,
 * over all tables, counted by the library's allocator (CT_ERR_ARG if
 * bytes_out is null). */
int ct_debug_guard_buffers(int on);
int ct_debug_check_guards(ct_table* ct, int poke, int64_t* changed_out);
int ct_debug_fail_alloc(int n);
int ct_debug_device_bytes(int64_t* bytes_out);

/* ---------------------------------------------------------------- misc -- */
/* ct_read_ceiling: measurement support, no counterpart in the paper. Launches
 * on cuda_stream one kernel that reads `bytes` of device memory at dev_buf
 * once, 128-bit loads not kept in L1, eight in flight per thread, four CTAs of
 * 256 threads per SM, and stores nothing the caller sees: the bandwidth one
 * launch of that size reaches, to set beside a propagation moving as many
 * bytes. With ms_out (host, nullable) the call records CUDA events on the
 * stream right before and after the launch, as ct_options.profile does for a
 * propagation, waits for the second and writes the interval in ms; without
 * it the call returns once the kernel is launched. dev_buf must be 16-byte
 * aligned and bytes a positive multiple of 16 (else CT_ERR_ARG). */
int ct_read_ceiling(const void* dev_buf, int64_t bytes, void* cuda_stream, float* ms_out);
const char* ct_last_error(void);
const char* ct_status_string(int status);
int ct_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CT_H */
