/* sfsim.h - C ABI of the GB300 Schroedinger-Feynman simulator of random grid
 * circuits (arXiv:1807.10749, "Quantum Supremacy Is Both Closer and Farther
 * than It Appears").
 *
 * The problem statement follows Section 2 and Section 3 of the paper: a
 * circuit on a qubit grid, a straight cut of the grid into two blocks, a set of
 * simulation paths (all of them, or a fraction f for fidelity ~ f) and a list of
 * requested bitstrings go in; the amplitudes <x|U|0...0> summed over the
 * selected paths come out.
 *
 * Conventions used by every call:
 *   - Qubit q of an R x C grid sits at row q / C, column q % C (row-major).
 *   - Bit q of a bitstring (uint64) is the measured value of qubit q.
 *   - Complex numbers are interleaved (re, im) doubles.
 *   - Every function returns an int status: SF_OK (0) or a negative SF_E*
 *     code. sf_last_error() returns the message of the calling thread's last
 *     failure. No C++ exception crosses this interface.
 *   - Inputs are copied during the call; the library never frees or keeps a
 *     caller pointer after it returns (except the server, which copies the
 *     submitted arrays). Output buffers are owned by the caller.
 *   - Device pointers (the *_device calls) are CUDA global-memory pointers of
 *     the current device; streams are cudaStream_t passed as void*.
 *   - Not thread-safe per object: a plan or a server handle must not be used
 *     by two threads at once. Different handles are independent.
 */
#ifndef SFSIM_H
#define SFSIM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SF_API __attribute__((visibility("default")))
#else
#define SF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SF_OK = 0,
  SF_EINVAL = -1,       /* bad argument: gate, qubit, cut, size, selection */
  SF_ENOMEM = -2,       /* host or device memory, or a budget too small */
  SF_ECUDA = -3,        /* a CUDA call failed (message in sf_last_error) */
  SF_ETIMEOUT = -4,     /* sf_server_wait: not finished within the timeout */
  SF_ECANCELLED = -5,   /* the request was cancelled */
  SF_EUNSUPPORTED = -6  /* valid input this build does not handle */
};

/* Gate kinds. Matrices (Section 1 gate set; Eq. 1 for CZ; Section 7 for iSWAP):
 *   SF_H = (1/sqrt2)[[1,1],[1,-1]]    SF_T = diag(1, e^{i pi/4})
 *   SF_X_HALF = 1/2 [[1+i,1-i],[1-i,1+i]]   SF_Y_HALF = 1/2 [[1+i,-1-i],[1+i,1+i]]
 *   SF_Z = diag(1,-1)   SF_S = diag(1,i)   SF_CZ = diag(1,1,1,-1)
 *   SF_ISWAP = |00><00| + i|01><10| + i|10><01| + |11><11|
 *   SF_U1: 2x2 from m[0..8); SF_U2: 4x4 from m[0..32), row-major, on the basis
 *   index 2*bit(q0) + bit(q1). */
enum sf_gate_kind { SF_H = 0, SF_X_HALF, SF_Y_HALF, SF_T, SF_Z, SF_S, SF_CZ, SF_ISWAP, SF_U1, SF_U2 };

typedef struct {
  int32_t cycle;   /* clock cycle; gates of one cycle act on disjoint qubits */
  int32_t kind;    /* sf_gate_kind */
  int32_t q0, q1;  /* qubits (q1 ignored for one-qubit kinds) */
  double m[32];    /* SF_U1 / SF_U2 entries (re, im interleaved) */
} sf_gate;

typedef struct sf_circuit sf_circuit;
typedef struct sf_plan sf_plan;
typedef struct sf_server sf_server;

/* Build a circuit on a rows x cols grid (n = rows*cols <= 64) from n_gates
 * gates in time order. Copies the gates. Fails with SF_EINVAL on a bad qubit,
 * kind, a two-qubit gate on one qubit, or two gates of one cycle sharing a
 * qubit. */
SF_API int sf_circuit_create(int rows, int cols, const sf_gate* gates, int64_t n_gates, sf_circuit** out);

/* Parse the text format (NUL-terminated): a 'grid R C' line, then
 * '<cycle> <name> <qubits> [reals]' lines, names h t x_1_2 y_1_2 z s cz iswap
 * u1 u2; '#' starts a comment. */
SF_API int sf_circuit_parse(const char* spec_text, sf_circuit** out);
SF_API int sf_circuit_info(const sf_circuit* c, int* rows, int* cols, int64_t* n_gates);
SF_API void sf_circuit_destroy(sf_circuit* c);

/* Cross-gate decompositions (Section 2 footnote, Section 3, Section 7). CZ
 * always uses Eq. 1 (P0 (x) I + P1 (x) Z, projector on the half-A qubit). */
enum { SF_DEC_SCHMIDT = 0, /* operator-Schmidt (SVD of the realigned matrix) */
       SF_DEC_BLOCK4 = 1   /* Eq. 4way: P0, P1, |0><1|, |1><0| on the A side */ };
enum { SF_EXEC_BATCHED = 0, /* path tree, batched launches, deferred last level */
       SF_EXEC_PLAIN = 1    /* every path from the prefix checkpoint alone */ };

typedef struct {
  uint64_t side_b_mask;      /* bit q set: qubit q in half B; 0 = automatic
                                straight cut (Section 8: minimise the larger
                                block, then the number of cross gates) */
  int32_t decomposition;     /* SF_DEC_* for non-CZ cross gates */
  int32_t select_prefix_bits;/* x_s of FRACTION selection; -1 = max(0, x-7) */
  int32_t tile_bits;         /* log2 amplitudes per tile (<= 13), 0 = per segment
                                12 or 13, whichever is estimated faster */
  int32_t fuse_bits;         /* log2 amplitudes per thread register block
                                (fusion width), 0 = tuned default */
  int32_t exec_mode;         /* SF_EXEC_* */
  int32_t defer_last_level;  /* 1 (default) / 0: fold the last branch level
                                into the gather when the circuit allows */
  int64_t hbm_budget_bytes;  /* device memory the executor may use, 0 = 75% of
                                free memory at plan time */
  int32_t batch_paths;       /* max leaf groups (finals) per launch, 0 = as many as
                                hold 2^30 amplitudes of both halves, halved until
                                the workspace fits the memory budget */
  int32_t run_bits;          /* log2 contiguous amplitudes per copy run (the
                                index bits every pass keeps active), 0 = per
                                segment the width (4 or 3) whose program moves
                                fewer bytes */
  int32_t jit;              /* 1 (default) = compile every pass of the plan into a
                               kernel of its own at plan time (NVRTC; plan creation
                               fails with SF_EUNSUPPORTED where NVRTC is missing),
                               0 = the generic pass kernel */
  int32_t split_last;       /* with the last level folded into the gather: 0 = plan
                               the level before it and the last segment as one
                               program (no node is written between them), 1 = two
                               programs with the node in between */
  int32_t fp32x2;           /* specialised kernels: 1 (default) = register stages
                               made only of H, X^1/2, Y^1/2 and phase groups keep
                               each complex amplitude in one FP32x2 register pair,
                               so a butterfly is one packed add per output; 0 =
                               scalar FP32 arithmetic */
  int32_t dense_finals;     /* with the last level folded into the gather: 0 = the
                               last pass of each half's final program writes only
                               the blocks of 2^g amplitudes (g = cut gates of the
                               folded level) that hold a requested bitstring, into
                               a compact buffer, when that is at most a quarter of
                               the half and fits the budget; 1 = always write the
                               whole final state */
  int32_t precision;        /* SF_PREC_*: how the cross-path sum accumulates */
  int32_t projector_side;   /* SF_PROJ_*: which half carries Eq. 1's projector */
  int32_t tile_buffers;     /* specialised kernels: shared-memory tile buffers per
                               CTA, 3 (load, compute and store each on a buffer of
                               its own) or 2 (half the memory, so a third CTA of
                               2^12-amplitude tiles fits on an SM); 0 = 2 for tiles
                               of up to 2^12 amplitudes, 3 above */
  int32_t cycle_segments;   /* 0 (default) = each gate runs in the segment of the
                               deepest branch level whose light cone holds it
                               (the gates a level's branch operators commute
                               with run once in the parent node, for all its
                               children); 1 = segments are the cycle ranges
                               between consecutive branch levels */
  int32_t reserved[2];
} sf_plan_opts;

/* Which half of a cut CZ carries the projector of Eq. 1. CZ is symmetric, so
 * CZ = P0 (x) I + P1 (x) Z = I (x) P0 + Z (x) P1 (A-side factor first); the
 * two readings give the same full path sum but different individual paths.
 *   SF_PROJ_A (default): the projector on the half-A qubit of every cut CZ.
 *   SF_PROJ_ALTERNATE: on the half-A qubit of the even-numbered cut gates and
 *     the half-B qubit of the odd-numbered ones (time order (cycle, lower
 *     qubit, higher qubit), numbered from 0). A projected qubit is a pinned
 *     index bit, so a branching level's pins are then shared by both halves
 *     and the passes after it touch fewer amplitudes in total. */
enum { SF_PROJ_A = 0, SF_PROJ_ALTERNATE = 1 };

/* Precision of the path sum (Section 2 footnote: single-precision states,
 * higher-precision accumulators). The half states are complex64 and each
 * path's product A_j[x_A] * B_j[x_B] is formed in FP32 in every mode.
 *   SF_PREC_F64: the products are added to FP64 sums, one final after another
 *     in path order, starting from the output (the default).
 *   SF_PREC_COMPENSATED: the same FP64 additions with Neumaier compensation;
 *     the compensation terms (16 bytes per bitstring of workspace) are added
 *     to the output at the end of the call.
 * In both modes the order of additions is fixed by the path order alone, so
 * a result does not depend on the memory budget, the batch size or the
 * requests it was batched with. */
enum { SF_PREC_F64 = 0, SF_PREC_COMPENSATED = 1 };

SF_API void sf_plan_opts_default(sf_plan_opts* o);

/* Plan the simulation: cut, cross gates (time order (cycle, lower qubit,
 * higher qubit)), decomposition, path tree, fused passes. When a CUDA device
 * is present, the plan's device state is set up on the current device here
 * (gather tables, the wait-timeout flag, the memory budget) and every kernel
 * the plan runs is loaded, so that later calls load no code. Without a device
 * the plan can still be inspected and sized (sf_plan_info, sf_workspace_size
 * with a budget, sf_selection_*). */
SF_API int sf_plan_create(const sf_circuit* c, const sf_plan_opts* opts, sf_plan** out);

/* n_cross: cross gates; path_bits: log2 of the path count (each cross gate
 * contributes log2 of its term count, 1 for CZ); m_a / m_b: half sizes;
 * n_levels: branching levels (cycles with cross gates). Any pointer may be
 * NULL. */
SF_API int sf_plan_info(const sf_plan* p, int* n_cross, int* path_bits, int* m_a, int* m_b, int* n_levels);

/* Planner statistics: passes per half over the whole circuit, register
 * stages, deferred gates at the last level. */
SF_API int sf_plan_stats(const sf_plan* p, int* passes_a, int* passes_b, int* stages_a, int* stages_b,
                  int* deferred);
/* Per-segment breakdown: segment 0 runs from the start to the first branch
 * level, segment s >= 1 from level s to the next; segment n_levels + 1 is
 * the last segment with its level folded into the gather (when it is).
 * half: 0 = A, 1 = B. passes/stages of that segment's program and its
 * algorithmic bytes for one node (live amplitudes read + written, 8 B). */
SF_API int sf_plan_segment_stats(const sf_plan* p, int half, int segment, int* passes, int* stages,
                                 double* bytes_per_node);
/* Human-readable description of the plan (cut, levels, and per segment and
 * half the passes: active bits, pins, register stages and their gates), in
 * the spirit of the per-run logs of the paper's appendices. Writes at most
 * cap bytes (NUL-terminated) and the full length to *len. */
SF_API int sf_plan_describe(const sf_plan* p, char* buf, size_t cap, size_t* len);
SF_API void sf_plan_destroy(sf_plan* p);

/* Path selection (Eq. 3; Section 3). Path ids number the branch choices, the
 * earliest cross gate in the most significant bits.
 *   SF_SEL_RANGE: ids first .. first+count-1.
 *   SF_SEL_FRACTION: K = max(1, floor(fidelity * 2^xs + 1e-9)) prefixes of xs
 *     bits, the images of 0..K-1 under the keyed Feistel permutation (key =
 *     seed), each with all its suffixes; xs = the plan's select_prefix_bits.
 *   SF_SEL_LIST: the n_list ids in list (any order, duplicates rejected). */
enum { SF_SEL_RANGE = 0, SF_SEL_FRACTION = 1, SF_SEL_LIST = 2 };
typedef struct {
  int32_t mode;
  uint64_t first, count;
  double fidelity;
  uint64_t seed;
  const uint64_t* list;
  int64_t n_list;
} sf_path_sel;

/* Autotuner (batching axis): times candidate plans of the circuit on the
 * first sample_paths paths of *sel (as a path list) for the n device
 * bitstrings d_bits - once to warm up, once timed with CUDA events on a
 * private stream - and writes the fastest candidate's options to *best, its
 * time to *best_seconds and the time of *base itself to *base_seconds (either
 * may be NULL). *base is always a candidate, so *best_seconds <= *base_seconds.
 * Stage 1 searches the pass shape on top of *base: tile_bits 0 (the planner's
 * per-segment choice, with run_bits 0), 12 or 13 with run_bits 3 or 4, each with
 * fusion width fuse_bits = k in {2, 3, 4, 5} register qubits per thread block
 * (k = 6 would need 64 amplitudes per thread: more registers than a thread of
 * the pass kernel holds). Stage 2 varies batch_paths, the leaf groups per
 * launch, over {1, 4, 16, 64, 256, 1024} at the best shape. With base->jit set
 * each candidate's specialised kernels are compiled before it is timed.
 * Allocates and frees the device memory it needs. */
SF_API int sf_plan_autotune(const sf_circuit* c, const sf_plan_opts* base, const sf_path_sel* sel,
                            int64_t sample_paths, const uint64_t* d_bits, int64_t n, sf_plan_opts* best,
                            double* best_seconds, double* base_seconds);

/* Runtime model of Section 8 (Eq. t_tot), with a fixed cost per request:
 *   T = C0 + C1 f 2^{x_p} (q1 2^{q1} + q2 2^{q2}) (d_p + C2 2^{x_b} d_b) + C3 P n_a
 * with q1, q2 the half sizes, x_p the selection prefix bits (select_prefix_bits),
 * x_b the path bits below them, f 2^{x_p} the selected prefixes, d_p the
 * cycles before the cycle of the last prefix cross gate, d_b the remaining
 * cycles, P the selected paths and n_a the bitstrings. C0 (launches, uploads,
 * the final copy) is not in the paper's equation. The model is linear:
 *   T = a . t,  a = (C0, C1, C1 C2, C3),
 * t = (1, f 2^{x_p} (q1 2^{q1} + q2 2^{q2}) d_p, f 2^{x_p} (...) 2^{x_b} d_b, P n_a).
 * sf_plan_cost_terms writes t (4 doubles) for a request (host only, no GPU
 * work). sf_cost_fit fits a (a >= 0, least squares on relative error) from n
 * requests' terms (4n doubles, row-major) and measured seconds; SF_EINVAL if
 * the set determines no coefficient. sf_cost_predict returns a . t. */
SF_API int sf_plan_cost_terms(const sf_plan* p, const sf_path_sel* sel, int64_t n_a, double* terms);
SF_API int sf_cost_fit(const double* terms, const double* seconds, int64_t n, double* coeffs);
SF_API double sf_cost_predict(const double* terms, const double* coeffs);

/* Number of selected paths and f_actual = selected / 2^path_bits. */
SF_API int sf_selection_size(const sf_plan* p, const sf_path_sel* sel, uint64_t* n_paths, double* f_actual);

/* Write the selected path ids in increasing order into ids[0..cap) (host).
 * *n_written = min(selected, cap). The enumeration the executor sums. */
SF_API int sf_selection_ids(const sf_plan* p, const sf_path_sel* sel, uint64_t* ids, uint64_t cap,
                     uint64_t* n_written);

/* Amplitudes, host buffers: out_amps[2*i], out_amps[2*i+1] = sum over the
 * selected paths of A_j[x_A] * B_j[x_B] for bitstrings[i] (Eq. 2 / Eq. 3, no
 * renormalisation by f). out_f_actual may be NULL. Allocates its device
 * memory inside the call (kept with the plan for the next call, freed by
 * sf_plan_drop_resident or sf_plan_destroy); blocks until done. When the
 * device has less free memory than the plan's budget assumed, the workspace
 * takes fewer finals per launch (same results); SF_ENOMEM when one does not
 * fit. */
SF_API int sf_amplitudes(sf_plan* p, const uint64_t* bitstrings, int64_t n, const sf_path_sel* sel,
                  double* out_amps, double* out_f_actual);

/* Device form: bytes of device workspace sf_amplitudes_device needs for n
 * bitstrings and this selection: the path-tree node buffers and, when the
 * plan writes compact finals (sf_plan_opts.dense_finals), the part maps and
 * compact buffers, which grow with n. Needs no device when the plan was
 * made with hbm_budget_bytes > 0. */
SF_API int sf_workspace_size(const sf_plan* p, int64_t n, const sf_path_sel* sel, size_t* bytes);

/* Device form: d_bitstrings (n uint64) and d_out_amps (2n doubles) are device
 * pointers; d_workspace of ws_bytes >= sf_workspace_size(). All work is
 * enqueued on cuda_stream; the call returns after the last launch is enqueued
 * and the result is valid once the stream reaches it. With accumulate != 0 the
 * sums are added to d_out_amps; otherwise d_out_amps is overwritten. Check
 * sf_plan_status once the stream is done: a kernel whose bounded wait gave
 * up leaves the result invalid.
 * Resident nodes: the plan leaves path-tree nodes in the workspace, and its
 * next call with the same workspace reuses those it needs (the path prefixes
 * that consecutive selections share, Section 2's checkpoints). The library
 * records which plan ran last in each workspace and reuses nothing after
 * another plan ran there; a caller that writes the workspace memory itself
 * between two calls of one plan must call sf_plan_drop_resident first. */
SF_API int sf_amplitudes_device(sf_plan* p, const uint64_t* d_bitstrings, int64_t n, const sf_path_sel* sel,
                         double* d_out_amps, int accumulate, void* d_workspace, size_t ws_bytes,
                         void* cuda_stream);

/* Several requests on one plan at once (Section 2: paths are independent, so
 * requests that share a circuit share its path tree). The union of the
 * requests' selected paths is evolved once: every pass launch carries the
 * nodes of all requests, and each request's bitstrings are gathered from the
 * finals it selected into its own output. Each request's result is bit for
 * bit the one sf_amplitudes_device gives it alone. All pointers in reqs are
 * device pointers (sel is host memory, read during the call). */
typedef struct {
  const uint64_t* d_bitstrings;  /* n uint64 */
  int64_t n;
  const sf_path_sel* sel;
  double* d_out_amps;            /* 2n doubles */
  int32_t accumulate;
} sf_request;
SF_API int sf_workspace_size_batch(const sf_plan* p, const sf_request* reqs, int n_req, size_t* bytes);
SF_API int sf_amplitudes_device_batch(sf_plan* p, const sf_request* reqs, int n_req, void* d_workspace,
                                      size_t ws_bytes, void* cuda_stream);

/* Status of the device forms: waits for cuda_stream, then reads and clears
 * the plan's wait-timeout flag. Every wait inside the pass kernels is bounded
 * (about 2^31 cycles); one that gives up sets this flag and ends its kernel,
 * which leaves the amplitudes of that call invalid. Returns SF_ECUDA if the
 * flag was set (or a timeout was injected, below), SF_OK otherwise. The host
 * forms (sf_amplitudes, sf_probabilities) and the server check the flag
 * themselves and return SF_ECUDA for the call or request concerned. */
SF_API int sf_plan_status(sf_plan* p, void* cuda_stream);

/* Forget the plan's resident nodes (its next device call recomputes every
 * node) and free the device buffers its host-form calls keep. */
SF_API int sf_plan_drop_resident(sf_plan* p);

/* Test hook (host side, nothing is run on the device): the next `count`
 * checks of a wait-timeout flag, in any form, report a timeout as if a
 * kernel had set the flag. count = 0 cancels pending injections. */
SF_API int sf_debug_inject_wait_timeouts(int count);
/* Test hook: writes `value` into the plan's device wait-timeout flag (as a
 * kernel that gave up would write 1), so the flag-reading path of every form
 * can be tested without a timeout on the device. Synchronous. */
SF_API int sf_debug_set_wait_flag(sf_plan* p, int value);

/* Probabilities (Section 3; Section 4 samples from them): p_i = |amp_i|^2,
 * divided by f_actual when divide_by_f != 0 (f_actual = selected paths /
 * all paths, the fidelity of a truncated path sum). Host form: as
 * sf_amplitudes, writing n doubles. Device form: probabilities of 2n-double
 * amplitudes d_amps into n doubles d_probs, times `scale`, computed in FP64
 * as (re*re + im*im) * scale in that order without contraction. */
SF_API int sf_probabilities(sf_plan* p, const uint64_t* bitstrings, int64_t n, const sf_path_sel* sel,
                            int divide_by_f, double* out_probs, double* out_f_actual);
SF_API int sf_probabilities_device(const double* d_amps, int64_t n, double scale, double* d_probs,
                                   void* cuda_stream);

/* Frugal rejection sampling, the accept step of Algorithm 2 (Section 4):
 * candidate j (a uniformly drawn bitstring whose amplitude is d_amps[2j],
 * d_amps[2j+1], e.g. the output of sf_amplitudes_device) is accepted iff
 *   d_uniform[j] < min(1, t_j),  t_j = ((re^2 + im^2) * prob_scale) * N / mprime
 * evaluated in FP64 in exactly this order without fused multiply-adds, so the
 * decision is reproducible on the host. N = 2^n (qubits), mprime = M' (10 in
 * the paper), prob_scale = 1, or 1/f_actual to renormalise a truncated path
 * sum. d_uniform: n doubles in [0, 1) supplied by the caller. d_accept: n
 * bytes, 1 = accepted; d_count: one int64, set to the number accepted. All
 * pointers are device pointers; the work is enqueued on cuda_stream. */
SF_API int sf_frugal_accept_device(const double* d_amps, const double* d_uniform, int64_t n, double N,
                                   double mprime, double prob_scale, uint8_t* d_accept, int64_t* d_count,
                                   void* cuda_stream);

/* Fidelity estimate between two sets of amplitudes on the same bitstrings
 * (Appendix C, the validation protocol; Section 3): with a = d_amps_a and
 * b = d_amps_b (2n doubles each, interleaved), writes to d_out (5 doubles,
 * device) Re and Im of sum_j conj(a_j) b_j, sum_j |a_j|^2, sum_j |b_j|^2,
 * accumulated in FP64, and the estimate f_e = |<a|b>|^2 / (<a|a> <b|b>)
 * (0 when a norm is zero). Enqueued on cuda_stream. */
SF_API int sf_overlap_device(const double* d_amps_a, const double* d_amps_b, int64_t n, double* d_out,
                             void* cuda_stream);

/* Fixed-scratch form of sf_amplitudes_device. This call has no counterpart
 * in the paper. It serves callers that must not allocate device memory once
 * they run: cudaMalloc may synchronise the device, and fails when another
 * allocator in the process (a framework's caching allocator, say) already
 * holds the free memory. The workspace that sf_amplitudes_device takes from
 * its caller - path-tree node buffers, compact-final maps and buffers, and
 * the compensation terms of SF_PREC_COMPENSATED - lives instead in one array
 * of SF_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library's module keeps until process exit. Arguments are those of
 * sf_amplitudes_device minus the workspace: d_bitstrings (n uint64) and
 * d_out_amps (2n doubles, overwritten unless accumulate != 0) are caller-owned
 * device buffers; the work is enqueued on cuda_stream.
 *   - The call never calls cudaMalloc, cudaFree or an allocating library
 *     routine, and loads no code: the plan must have been created with this
 *     device current (sf_plan_create then allocates the plan's gather tables
 *     and wait-timeout flag, loads every kernel the plan runs and looks up the
 *     array's device address with cudaGetSymbolAddress). Otherwise SF_EINVAL.
 *   - A plan and request whose workspace would exceed the array are rejected
 *     with SF_ENOMEM and a message naming the bytes needed.
 *   - All calls share the one array, which keeps the previous call's
 *     contents (every byte a call reads it has written first, and the
 *     compensation terms are zeroed per call); calls that can overlap on the
 *     GPU (other streams, other threads) race on it and must be serialised by
 *     the caller.
 *   - Results equal sf_amplitudes_device's bit for bit. A wait timeout is
 *     reported by sf_plan_status, as for the device form. */
#define SF_NOALLOC_SCRATCH_BYTES (64ull << 20)
SF_API int sf_amplitudes_device_noalloc(sf_plan* p, const uint64_t* d_bitstrings, int64_t n,
                                        const sf_path_sel* sel, double* d_out_amps, int accumulate,
                                        void* cuda_stream);

/* Request server (continuous batching): requests are admitted while their
 * device footprint fits hbm_budget_bytes; admitted requests run concurrently
 * on their own streams. Each request's result equals sf_amplitudes on the same
 * input. A worker whose workspace allocation fails for lack of free memory
 * lays it out with fewer finals per launch. */
SF_API int sf_server_create(int64_t hbm_budget_bytes, int max_concurrent, sf_server** out);
/* Copies bitstrings and the selection's list. The plan must outlive the
 * request. */
SF_API int sf_server_submit(sf_server* s, sf_plan* p, const uint64_t* bitstrings, int64_t n,
                     const sf_path_sel* sel, uint64_t* ticket);
/* Waits up to timeout_ms (<0: forever). On SF_OK copies 2n doubles into
 * out_amps and releases the ticket; SF_ETIMEOUT keeps it. */
SF_API int sf_server_wait(sf_server* s, uint64_t ticket, int timeout_ms, double* out_amps);
/* Cancels a queued or running request; its wait returns SF_ECANCELLED. */
SF_API int sf_server_cancel(sf_server* s, uint64_t ticket);
/* Seconds from submit to admission and to completion of a finished ticket
 * (before its wait), for latency reports. */
SF_API int sf_server_times(sf_server* s, uint64_t ticket, double* queued_s, double* total_s);
/* Admission by the runtime model (Section 8, Eq. t_tot): with coeffs (C0,
 * C1, C1 C2, C3 as sf_cost_fit returns them) set, among the requests that fit the
 * budget the one with the shortest predicted time is admitted first; a
 * request queued longer than max_wait_s seconds goes before all others (in
 * arrival order) and, if it does not fit, blocks admission until memory
 * frees. coeffs = NULL restores arrival order. */
SF_API int sf_server_set_cost_model(sf_server* s, const double* coeffs, double max_wait_s);
/* Batches the server has run and the requests in them (a batch holds the
 * queued requests of one plan, run together). Any pointer may be NULL. */
SF_API int sf_server_stats(sf_server* s, int64_t* batches, int64_t* requests, int64_t* max_batch);
SF_API void sf_server_destroy(sf_server* s);

/* Kernel counters of one plan, for roofline reports. sf_plan_profile resets
 * them and turns per-launch CUDA-event timing on (enable_timing = 1) or off.
 * sf_plan_profile_read returns, for kernel 0 (fused tile pass), 1 (gather)
 * or 2 (other), the launches since the reset, their summed device time in
 * seconds (0 unless timing was on; blocks until those launches finished)
 * and their algorithmic bytes (state amplitudes read + written, 8 bytes each,
 * for passes, where a compact final pass counts the parts it writes;
 * bitstrings, gathered amplitudes and accumulators for gathers). Reading
 * waits for the device when compact final passes were counted. */
SF_API int sf_plan_profile(sf_plan* p, int enable_timing);
SF_API int sf_plan_profile_read(sf_plan* p, int kernel, int64_t* launches, double* seconds, double* bytes);

SF_API const char* sf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SFSIM_H */
