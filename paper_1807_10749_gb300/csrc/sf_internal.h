// Internal structures of the sfsim library: circuit, plan (cut, cross-gate
// terms, path tree levels, fused pass programs) and the device launch records.
#pragma once

#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sfsim.h"

namespace sf {

using cd = std::complex<double>;

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
struct Error {
  int code;
  std::string msg;
};
[[noreturn]] void fail(int code, const std::string& msg);

// ----------------------------------------------------------------- circuit
struct Gate {
  int cycle = 0;
  int kind = 0;
  int q0 = 0, q1 = -1;
  cd m[16];  // 2x2 (first 4) or 4x4, row-major; basis 2*bit(q0)+bit(q1)
  int nq() const { return (kind == SF_CZ || kind == SF_ISWAP || kind == SF_U2) ? 2 : 1; }
};

struct Circuit {
  int rows = 0, cols = 0, n = 0;
  std::vector<Gate> gates;  // stable-sorted by cycle
};

void gate_matrix(Gate& g);  // fills g.m for named kinds
Circuit* circuit_from_gates(int rows, int cols, const sf_gate* gates, int64_t n_gates);
Circuit* circuit_parse(const char* text);

// ------------------------------------------------------------------ linalg
// One-sided Jacobi SVD of a complex 4x4 matrix: R = U diag(s) V^H, s
// descending.
void svd4(const cd R[16], cd U[16], double s[4], cd V[16]);

}  // namespace sf

#include "dev_types.h"

namespace sf {

// Gather: per bitstring, sum over the launch's finals of the (deferred)
// contraction, added to acc in FP64.
struct GatherFinal {
  const void* wa;  // float2*
  const void* wb;
  uint64_t path;   // digits for pins and leaf lists (group id << defer bits)
  double sre, sim; // complex scale of this final (sigma_A * sigma_B)
  int32_t all_leaves;         // 1: every leaf of the deferred level
  uint64_t leafmask[4];       // else: selected leaf digits (bit b = leaf b)
};

// Compact finals (PassLaunch::cmap): amplitude j of a final sits at
// slot(P) * 2^ctl + (j mod 2^ctl), P = (pext(j, cfree) << ckt) | pext(j, cpart)
// its part; a block of the gather spans one part, or two when csub1 != 0
// (position ctl is then a block bit; csub1 is its contribution to P).
struct CompactMap {
  const uint32_t* cmap;  // null: dense
  uint32_t cfree;        // free positions of the final pass
  uint32_t cpart;        // its active positions from ctl up
  int32_t ckt, ctl;      // k - ctl, ctl
  uint32_t csub1;
};

struct GatherSide {
  CompactMap c;
  int32_t npin;
  DevPin pin[MAX_PINS];
  int8_t dpos[MAX_DEFER];  // layout positions of the deferred qubits
  int8_t dq[MAX_DEFER];    // their global qubit numbers (bits of x)
};

struct GatherLaunch {
  const uint32_t* tabA;  // 8 x 256 byte tables: x byte -> layout index part
  const uint32_t* tabB;
  const uint64_t* bits;
  double* acc;           // 2n doubles; every final's term is added to it in order
  double* comp;          // null, or 2n compensation terms (SF_PREC_COMPENSATED)
  int64_t n;
  int32_t g;             // deferred gates
  int32_t nterm_bits;    // log2 terms per deferred gate (1 or 2)
  GatherSide A, B;
  float ma[MAX_DEFER][4][8];  // M^A_{i,d} = V^A_i F^A_{i,d}, 2x2 interleaved
  float mb[MAX_DEFER][4][8];
  uint8_t xshift[MAX_CROSS];
  uint8_t xbits[MAX_CROSS];
  int32_t n_finals;
  GatherFinal finals[GATHER_FINALS];
};

// -------------------------------------------------------------- host plan
struct Pin {
  int pos;  // half layout position
  int xi;   // -1 const
  int v[4];
};

// Host-side op of a half (positions are layout positions).
enum HopKind { H_G1, H_G2, H_CZ, H_PHASE1, H_DMUL, H_XSEL, H_XPHASE, H_PROJ };
struct HOp {
  int kind = -1;
  int p0 = -1, p1 = -1;
  int fast = 0;       // DOP_H / DOP_XH / DOP_YH for H_G1 with that matrix
  int scale_e = 0;    // deferred factor (1/sqrt2)^scale_e of the fast form
  int w = 0;          // H_PHASE1: weight (mod 8) of e^{i pi/4}
  cd m[16];           // matrix (G1: 4, G2: 16, DMUL: 2 diag)
  int xi = -1;        // cross gate index for X* ops
  int nterm = 0;
  cd tm[4][4];        // per-digit 2x2 factor (XSEL), or diag (XPHASE uses tw)
  int tw[4] = {0, 0, 0, 0};  // XPHASE weights per digit
  int pv[4] = {0, 0, 0, 0};  // PROJ kept value per digit
  bool diag() const { return kind == H_CZ || kind == H_PHASE1 || kind == H_DMUL || kind == H_XPHASE; }
};

struct PassPlan {
  int jit_id = -1;  // index into Plan::jit_entries (specialised kernel), -1 = generic
  DevPass dev;
  std::vector<DevStage> stages;
  std::vector<DevOp> ops;
  std::vector<DevPhaseGroup> phases;
  std::vector<float> mats;
};

struct SegmentPlan {
  std::vector<PassPlan> passes;
  std::vector<Pin> pins_out;  // pins of the segment's output
  cd scale = 1.0;             // sigma: true = scale * stored (relative to input)
  int n_stages = 0;
};

struct HalfPlan {
  int m = 0;
  std::vector<int> qubits;    // global qubit at layout position p
  std::vector<int> pos_of;    // global qubit -> layout position (-1 if not here)
  std::vector<std::vector<HOp>> seg_ops;  // per segment
  std::vector<Pin> root_pins; // root input pins (qubits without leading H)
  cd root_scale = 1.0;
  std::vector<SegmentPlan> seg;          // per segment, full program
  SegmentPlan last_deferred;             // last segment without deferred ops
  SegmentPlan last_merged;               // the level before it and last_deferred as one program
  std::vector<uint32_t> tab;             // 8 x 256 gather byte tables
};

struct CrossGate {
  int gate_index;
  int cycle;
  int qa, qb;     // global qubits on side A / B
  int nterm;      // power of two
  int bits;
  int shift;      // path-id bit offset of its digit
  cd fa[4][4], fb[4][4];  // per-term 2x2 factors
};

struct Level {
  int cycle;
  int first_cross, n_cross;
  int bits;   // total bits of the level
  int shift;  // lowest path bit of the level
};

// Kernel counters (sf_plan_profile): launches, algorithmic bytes, and, when
// timing is on, CUDA events around each launch.
struct ProfRec {
  int kind;
  void* e0;  // cudaEvent_t
  void* e1;
};
// Bytes known on the device only (the compact final writes: requested blocks
// x bytes per block), read back when the profile is collected.
struct ProfUnits {
  int kind;
  const uint32_t* count;  // device counter
  double unit;            // bytes per count
};
struct Profile {
  bool timing = false;
  int64_t launches[3] = {0, 0, 0};
  double bytes[3] = {0, 0, 0};
  double seconds[3] = {0, 0, 0};
  std::vector<ProfRec> pending;
  std::vector<ProfUnits> units;
  std::vector<void*> pool;
};
constexpr int kCountRing = 1024;  // calls whose block counts the profile can hold

struct Plan {
  sf_plan_opts opts;
  Profile prof;
  Circuit circ;
  uint64_t side_b_mask = 0;
  std::vector<CrossGate> cross;
  std::vector<Level> levels;
  int path_bits = 0;
  int xs = 0;  // FRACTION prefix bits
  HalfPlan A, B;
  bool deferred = false;       // last level folded into the gather
  bool merged_last = false;    // finals run last_merged from depth nL - 2 (no depth nL - 1 nodes)
  int defer_bits = 0;          // bits of the last level when deferred
  float ma[MAX_DEFER][4][8];
  float mb[MAX_DEFER][4][8];
  int tile_bits = 13, fuse_bits = 5, run_bits = 3;
  // device copies
  uint32_t* d_tabA = nullptr;
  uint32_t* d_tabB = nullptr;
  int* d_err = nullptr;  // device error flag of bounded waits
  uint32_t* d_cnt = nullptr;  // requested-block counts per call and half (kCountRing x 2)
  uint64_t cnt_seq = 0;
  int device = 0;
  // executor cache (resident nodes between calls that reuse a workspace)
  void* cache = nullptr;
  // specialised pass kernels (opts.jit): compiled-kernel cache entries
  std::vector<void*> jit_entries;
};

Plan* plan_create(const Circuit& c, const sf_plan_opts& o);
std::string plan_describe(const Plan& p);
void plan_destroy(Plan* p);

// ------------------------------------------------------------- selection
struct Range {
  uint64_t lo, hi;  // [lo, hi)
};
// Sorted, disjoint ranges of selected path ids.
std::vector<Range> select_ranges(const Plan& p, const sf_path_sel& s, double* f_actual);
uint64_t feistel(uint64_t v, int w, uint64_t key);

// -------------------------------------------------------------- executor
// Per-call context: where the resident-node cache lives, whether launches are
// counted in the plan's profile, and a cancellation flag checked between
// path blocks. nullptr = the plan's own cache and profile, no cancellation.
struct ExecCtx {
  void** cache_slot = nullptr;
  bool profile = true;
  const volatile int* cancel = nullptr;  // single-request form
  int* err = nullptr;                    // error flag to use instead of the plan's
  int64_t budget = 0;                    // memory budget instead of the plan's
};
// One request of a batch on one plan: its bitstrings, selection (ranges),
// output and cancellation flag.
struct ExecReq {
  const uint64_t* d_bits = nullptr;
  int64_t n = 0;
  std::vector<Range> rs;
  double* d_out = nullptr;
  int accumulate = 0;
  const volatile int* cancel = nullptr;
  bool cancelled = false;  // set by exec_run
};
size_t exec_workspace_bytes(const Plan& p, int64_t n, const sf_path_sel& s, int64_t budget = 0);
size_t exec_workspace_bytes(const Plan& p, const std::vector<ExecReq>& reqs, int64_t budget = 0);
// cudaMalloc of a workspace for reqs, with fewer finals per launch when the
// device's free memory is short; returns the layout budget used.
int64_t exec_alloc_workspace(const Plan& p, const std::vector<ExecReq>& reqs, int64_t budget, void** ws,
                             size_t* bytes);
void exec_run(Plan& p, const uint64_t* d_bits, int64_t n, const sf_path_sel& s, double* d_out,
              int accumulate, void* ws, size_t ws_bytes, void* stream, bool keep_cache,
              ExecCtx* ctx = nullptr);
// The union of the requests' paths evolved once, each request gathered into
// its own output; fails with SF_ECANCELLED only when every request is
// cancelled (the others' results are then complete).
void exec_run(Plan& p, std::vector<ExecReq>& reqs, void* ws, size_t ws_bytes, void* stream, bool keep_cache,
              ExecCtx* ctx = nullptr);
void exec_free_cache(void* cache);
void exec_forget_workspace(const void* ws);  // no cache may reuse nodes left in ws

// Features of the runtime model (Section 8, Eq. t_tot) for a request.
void cost_terms(const Plan& p, const sf_path_sel& s, int64_t n_a, double t[4]);

// Run-time specialised pass kernels (jit.cpp).
void jit_prepare(Plan& p);
void jit_load(Plan& p);  // load the plan's specialised kernels on the current device
// The fixed scratch of sf_amplitudes_device_noalloc: its device address on
// `device` (looked up once, with that device current).
void* noalloc_prepare(int device);
// Waits for the stream, reads and clears a wait-timeout flag; fails with
// SF_ECUDA if it was set or a timeout was injected (sf_debug_inject_wait_timeouts).
void check_wait_flag(int* d_flag, void* stream);
std::string jit_source(const PassPlan& pp);
void launch_pass_jit(const PassLaunch& L, int tiles, void* entry, void* stream);
void ensure_device(Plan& p);
void exec_release_cache(Plan& p);
double segment_bytes(const SegmentPlan& s);  // algorithmic bytes of one node
void prof_begin(Plan& p, int kind, double bytes, void* stream, void** e1_out, int launches = 1);
void prof_end(Plan& p, void* e1, void* stream);
void prof_collect(Plan& p);
void prof_release(Plan& p);

// ---------------------------------------------------------------- kernels
void launch_pass(const PassLaunch& L, int tiles, int fuse_bits, int tile_bits, void* stream);
void launch_gather(const GatherLaunch& L, void* stream);
// Part maps of the compact finals (PassLaunch::cmap) for n bitstrings: per
// half with map != null, zero the map, mark the parts of every bitstring's
// block, then fill the per-word prefix counts (sums: scratch of
// ceil(nw / 2048) words) and write the number of marked parts to count
// (unless null).
struct BlockMapLaunch {
  const uint32_t* tab[2];
  const uint64_t* bits;
  int64_t n;
  CompactMap c[2];   // c[s].cmap unused here: map[s] is written
  uint32_t* map[2];
  int64_t nw[2];
  uint32_t* sums[2];
  uint32_t* count[2];
};
// Marks the parts of every set of bitstrings (L.bits / L.n are replaced by
// each set in turn); returns kernels launched.
int launch_block_maps(const BlockMapLaunch& L, const std::vector<std::pair<const uint64_t*, int64_t>>& sets,
                      void* stream);
void launch_zero(double* p, int64_t n_doubles, void* stream);
void launch_fold(double* out, const double* comp, int64_t n_doubles, void* stream);
void launch_prob(const double* amps, int64_t n, double scale, double* probs, void* stream);
void launch_overlap(const double* a, const double* b, int64_t n, double* out, void* stream);  // out: 5 doubles
void preload_kernels();  // load every static kernel into the current context
void launch_frugal(const double* amps, const double* u, int64_t n, double N, double mp, double scale,
                   uint8_t* acc, int64_t* count, void* stream);

}  // namespace sf

// Handle types of the C ABI (shared by capi.cpp and server.cpp).
struct sf_circuit {
  sf::Circuit c;
};

struct SfHostBuffers {  // device buffers of the host-pointer call, reused
  void* ws = nullptr;
  size_t ws_bytes = 0;
  uint64_t* bits = nullptr;
  double* out = nullptr;   // 3 cap_n doubles: amplitudes, then probabilities
  int64_t cap_n = 0;
  void* stream = nullptr;  // cudaStream_t
  double* probs(int64_t n) { (void)n; return out + 2 * cap_n; }
};

struct sf_plan {
  sf::Plan* p = nullptr;
  SfHostBuffers hb;
};
