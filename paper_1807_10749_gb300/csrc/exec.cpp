// Executor: walks the selected paths as a tree (Section 2: a process owns a
// path prefix, checkpoints its state and runs every suffix from it; here the
// checkpoints are resident device buffers per tree depth), launches the fused
// passes for all nodes of a depth together, and gathers the requested
// amplitudes of each batch of finished paths into FP64 sums (Eq. 2 / Eq. 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <unordered_map>

#include "sf_internal.h"

namespace sf {

namespace {

size_t node_bytes(const Plan& p) { return (((size_t)1 << p.A.m) + ((size_t)1 << p.B.m)) * 8; }

struct Slot {
  uint64_t id = ~0ull;
  bool valid = false;
  bool dead = false;
  cd sa = 1.0, sb = 1.0;
};

struct Cache {
  const void* ws = nullptr;
  size_t ws_bytes = 0;
  int B = 0;
  std::vector<int> cap;                    // per cached depth
  std::vector<size_t> first_slot;          // per cached depth
  std::vector<std::vector<Slot>> slots;    // per cached depth
  size_t final_first = 0;
};

struct Final {
  uint64_t fid;
  bool all;
  uint64_t mask[4];
};

int total_bits_below(const Plan& p, int depth) {  // bits of levels[depth .. nL-1]
  int b = 0;
  for (size_t l = depth; l < p.levels.size(); l++) b += p.levels[l].bits;
  return b;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Compact finals. With the last level folded into the gather, the gather
// reads from each final only the blocks of 2^g amplitudes (the g cut qubits
// of the folded level sit at layout positions 0..g-1) that hold a requested
// bitstring. The last pass of a half's final program then writes just those
// blocks' parts (a part is a tile's share of a block: positions 0..ctl-1 of
// the tile), into a compact buffer, when that buffer is at most a quarter of
// the half. The parts are numbered tile-major (PassLaunch::cmap), so a tile
// reads its stretch of the part map with one coalesced load. A half
// qualifies when that pass has no output pins (every tile is written, none
// pinned away), its lowest ctl >= 1 tile bits are positions 0..ctl-1 and a
// block spans at most two parts (g - ctl <= 1).
struct CompactSide {
  bool on = false;
  CompactMap c{};    // without the map pointer
  size_t nw = 0;     // map words (32 parts each)
  size_t cap = 0;    // slots per final: min(parts of n blocks, parts)
  size_t map_bytes = 0, sums_bytes = 0, buf_bytes = 0;
};
struct Compact {
  int g = 0;
  CompactSide s[2];
  size_t fixed = 0;      // maps and chunk counts
  size_t per_final = 0;  // compact buffers of one final, both halves
  bool any() const { return s[0].on || s[1].on; }
};

const SegmentPlan& final_segment(const Plan& p, int side) {
  const HalfPlan& H = side ? p.B : p.A;
  return p.merged_last ? H.last_merged : (p.deferred ? H.last_deferred : H.seg[p.levels.size()]);
}

Compact compact_plan(const Plan& p, int64_t n) {
  Compact c;
  if (!p.deferred || p.opts.dense_finals || n <= 0 || p.levels.empty()) return c;
  const Level& lv = p.levels.back();
  const int g = lv.n_cross;
  if (g < 1 || g > MAX_DEFER) return c;
  c.g = g;
  for (int side = 0; side < 2; side++) {
    const HalfPlan& H = side ? p.B : p.A;
    const SegmentPlan& fin = final_segment(p, side);
    CompactSide& cs = c.s[side];
    if (fin.passes.empty() || !fin.pins_out.empty() || H.m <= g || H.m > 32) continue;
    const DevPass& d = fin.passes.back().dev;
    if (d.n_pin_out != 0 || d.n_free != H.m - d.k) continue;
    uint32_t dmask = 0;
    for (int t = 0; t < g; t++) {
      const CrossGate& x = p.cross[lv.first_cross + t];
      const int pos = H.pos_of[side ? x.qb : x.qa];
      if (pos >= 0 && pos < 32) dmask |= 1u << pos;
    }
    if (dmask != (1u << g) - 1u) continue;
    int tl = 0;
    while (tl < d.k && d.gpos[tl] < g) {
      if (d.gpos[tl] != tl) break;
      tl++;
    }
    if (tl < 1 || (tl < d.k && d.gpos[tl] < g) || g - tl > 1) continue;
    uint32_t active = 0;
    for (int j = 0; j < d.k; j++) active |= 1u << d.gpos[j];
    const uint32_t all = H.m == 32 ? 0xffffffffu : ((1u << H.m) - 1u);
    cs.c.cfree = all & ~active;
    cs.c.cpart = active & ~((1u << tl) - 1u);
    cs.c.ckt = d.k - tl;
    cs.c.ctl = tl;
    cs.c.csub1 = g > tl ? (pext32(1u << tl, cs.c.cfree) << cs.c.ckt) : 0u;
    const size_t parts = (size_t)1 << (H.m - tl);
    cs.cap = std::min<size_t>((size_t)n * (g > tl ? 2 : 1), parts);
    if ((cs.cap << tl) * 4 > ((size_t)1 << H.m)) continue;
    cs.on = true;
    cs.nw = (parts + 31) / 32;
    cs.map_bytes = align256(cs.nw * 8);
    cs.sums_bytes = align256(((cs.nw + 2047) / 2048) * 4);
    cs.buf_bytes = align256((cs.cap << tl) * 8);
    c.fixed += cs.map_bytes + cs.sums_bytes;
    c.per_final += cs.buf_bytes;
  }
  return c;
}

// The block size (finals per block) and per-depth slot capacities.
struct Layout {
  int B = 1;
  std::vector<int> cap;
  size_t total_slots = 0;
  bool compact = false;  // finals written as compact blocks (Compact)
  size_t bytes = 0;      // workspace bytes after alignment of its base
};

// Depths whose nodes are cached: all levels, except that the finals of a
// merged last program start from depth nL - 2.
int cached_depths(const Plan& p) {
  const int nL = (int)p.levels.size();
  return p.merged_last ? nL - 1 : nL;
}

// Bytes at the end of the workspace for the pass kernels' work counters.
constexpr size_t kWorkBytes = 256;

// extra: fixed bytes after the rest (the compensation terms of
// SF_PREC_COMPENSATED), counted against the budget; the work counters
// follow them.
Layout make_layout(const Plan& p, uint64_t n_finals, const Compact& cp, int64_t budget_override = 0,
                   size_t extra = 0) {
  extra += kWorkBytes;
  const int nL = cached_depths(p);
  const size_t nb = node_bytes(p);
  int64_t budget = budget_override > 0 ? budget_override : p.opts.hbm_budget_bytes;
  const size_t amps = ((size_t)1 << p.A.m) + ((size_t)1 << p.B.m);
  // default: finals of 2^30 amplitudes (both halves) per launch, halved below
  // until the layout fits the budget (7x8: 2, 5x10: 16)
  int64_t B = p.opts.batch_paths > 0 ? p.opts.batch_paths : std::max<int64_t>(1, ((int64_t)1 << 30) / (int64_t)amps);
  B = std::min<int64_t>(B, std::max<uint64_t>(1, n_finals));
  Layout lay;
  while (true) {
    lay.cap.assign(std::max(0, nL), 0);
    size_t tot = (size_t)B;
    int cum = 0;
    for (int s = 0; s < nL; s++) {
      int64_t c = (cum >= 62) ? B : std::min<int64_t>(B, (int64_t)1 << cum);
      lay.cap[s] = (int)c;
      tot += (size_t)c;
      if (s < nL) cum += p.levels[s].bits;
    }
    // compact finals when they fit: smaller blocks first, dense finals last
    const size_t dense = align256(tot * nb) + extra;
    const size_t withc = align256(tot * nb) + cp.fixed + (size_t)B * cp.per_final + extra;
    const bool fits_c = cp.any() && (int64_t)withc <= budget;
    if (fits_c || (!cp.any() && (int64_t)dense <= budget) || B == 1) {
      lay.B = (int)B;
      lay.total_slots = tot;
      lay.compact = fits_c;
      lay.bytes = fits_c ? withc : dense;
      if ((int64_t)lay.bytes > budget)
        fail(SF_ENOMEM, "device memory budget too small for one path (" + std::to_string(dense) +
                            " bytes needed)");
      return lay;
    }
    B = std::max<int64_t>(1, B / 2);
  }
}

uint64_t count_finals(const Plan& p, const std::vector<Range>& rs) {
  const int fb = p.deferred ? p.defer_bits : 0;
  uint64_t n = 0, last = ~0ull;
  for (auto& r : rs) {
    uint64_t a = r.lo >> fb, b = (r.hi - 1) >> fb;
    n += b - a + 1;
    if (a == last) n--;
    last = b;
  }
  return n;
}

void fill_launch(PassLaunch& L, const PassPlan& pp, const Plan& plan, int* err, uint32_t* work) {
  static_assert(sizeof(PassLaunch) <= 32764, "kernel parameter block too large");
  if (pp.stages.size() > (size_t)MAX_STAGES || pp.ops.size() > (size_t)MAX_OPS ||
      pp.phases.size() > (size_t)MAX_PHASE_GROUPS || pp.mats.size() > (size_t)2 * MAX_MATS)
    fail(SF_EUNSUPPORTED, "internal: pass program too large");
  L.pass = pp.dev;
  L.err = err;
  L.work = work;
  L.cmap = nullptr;
  L.ctl = L.cpad = 0;
  std::copy(pp.stages.begin(), pp.stages.end(), L.stages);
  std::copy(pp.ops.begin(), pp.ops.end(), L.ops);
  std::copy(pp.phases.begin(), pp.phases.end(), L.phases);
  std::copy(pp.mats.begin(), pp.mats.end(), L.mats);
  for (size_t i = 0; i < plan.cross.size(); i++) {
    L.xshift[i] = (uint8_t)plan.cross[i].shift;
    L.xbits[i] = (uint8_t)plan.cross[i].bits;
  }
}

int resolve(const Pin& pin, const Plan& p, uint64_t path) {
  if (pin.xi < 0) return pin.v[0];
  const CrossGate& x = p.cross[pin.xi];
  int d = (int)((path >> x.shift) & ((1u << x.bits) - 1));
  return pin.v[d];
}

bool dead_by_pins(const DevPass& dp, const Plan& p, uint64_t path) {
  for (int i = 0; i < dp.n_pin_in; i++)
    for (int j = i + 1; j < dp.n_pin_in; j++)
      if (dp.pin_in[i].pos == dp.pin_in[j].pos) {
        Pin a{dp.pin_in[i].pos, dp.pin_in[i].xi, {dp.pin_in[i].v[0], dp.pin_in[i].v[1], dp.pin_in[i].v[2], dp.pin_in[i].v[3]}};
        Pin b{dp.pin_in[j].pos, dp.pin_in[j].xi, {dp.pin_in[j].v[0], dp.pin_in[j].v[1], dp.pin_in[j].v[2], dp.pin_in[j].v[3]}};
        if (resolve(a, p, path) != resolve(b, p, path)) return true;
      }
  return false;
}

// The live part of a pass's input a node reads: its pins' values (bit i =
// value of input pin i). Nodes with one input buffer and equal keys read the
// same amplitudes.
uint64_t pin_key(const DevPass& dp, const Plan& p, uint64_t path) {
  uint64_t k = 0;
  for (int i = 0; i < dp.n_pin_in && i < 64; i++) {
    Pin a{dp.pin_in[i].pos, dp.pin_in[i].xi, {dp.pin_in[i].v[0], dp.pin_in[i].v[1], dp.pin_in[i].v[2], dp.pin_in[i].v[3]}};
    if (resolve(a, p, path)) k |= 1ull << i;
  }
  return k;
}

struct Job {
  const void* in;  // parent buffer (half base) or nullptr for generated input
  void* out;
  uint64_t path;
};

// Algorithmic bytes of one pass launch: live input amplitudes read (unless
// generated) once per distinct input buffer, plus live output amplitudes
// written per node (unless the writes are compact: counted on the device),
// 8 bytes each.
double pass_bytes(const DevPass& d, int nodes, int inputs, bool dense_out = true) {
  uint32_t active = 0;
  for (int j = 0; j < d.k; j++) active |= 1u << d.gpos[j];
  uint32_t pin_in = 0, pin_out = 0;
  for (int i = 0; i < d.n_pin_in; i++) pin_in |= 1u << d.pin_in[i].pos;
  for (int i = 0; i < d.n_pin_out; i++) pin_out |= 1u << d.pin_out[i].pos;
  const double tiles = std::ldexp(1.0, d.n_free);
  const double rd = d.gen_input ? 0.0 : tiles * std::ldexp(1.0, d.k - __builtin_popcount(pin_in & active));
  const double wr = tiles * std::ldexp(1.0, d.k - __builtin_popcount(pin_out & active));
  return 8.0 * (rd * inputs + (dense_out ? wr * nodes : 0.0));
}

// The compact output of a final program's last pass (per job: its buffer).
struct CompactOut {
  const uint32_t* cmap = nullptr;
  int ctl = 0;
  const uint32_t* count = nullptr;  // device count of marked parts (profile)
  std::vector<void*> out;
};

// Run a segment program for a batch of nodes of one half.
void run_segment(Cache&, Plan& plan, const SegmentPlan& seg, const std::vector<Job>& jobs,
                 cudaStream_t st, bool prof, int* err, uint32_t* work, const CompactOut* co = nullptr) {
  if (jobs.empty()) return;
  if (co && co->out.size() != jobs.size()) fail(SF_EINVAL, "internal: compact outputs");
  for (size_t p = 0; p < seg.passes.size(); p++) {
    const bool compact = co && p + 1 == seg.passes.size();
    const PassPlan& pp = seg.passes[p];
    static thread_local std::unique_ptr<PassLaunch> scratch;
    if (!scratch) {
      scratch = std::make_unique<PassLaunch>();
      std::memset(scratch.get(), 0, sizeof(PassLaunch));
    }
    PassLaunch* L = scratch.get();
    fill_launch(*L, pp, plan, err, work);
    if (compact) {
      L->cmap = co->cmap;
      L->ctl = co->ctl;
    }
    const int tiles = 1 << pp.dev.n_free;
    for (size_t j0 = 0; j0 < jobs.size(); j0 += MAX_NODES) {
      size_t j1 = std::min(jobs.size(), j0 + MAX_NODES);
      L->n_nodes = (int)(j1 - j0);
      for (size_t j = j0; j < j1; j++) {
        L->nodes[j - j0].in = (p == 0) ? jobs[j].in : jobs[j].out;
        L->nodes[j - j0].out = compact ? co->out[j] : jobs[j].out;
        L->nodes[j - j0].path = jobs[j].path;
      }
      void* e1 = nullptr;
      if (prof) {
        // siblings share their parent's buffer: count each input once (they
        // read disjoint pinned parts when pins separate them, so count those
        // as separate reads)
        std::vector<std::pair<const void*, uint64_t>> ins;
        for (int j = 0; j < L->n_nodes; j++) ins.push_back({L->nodes[j].in, pin_key(pp.dev, plan, L->nodes[j].path)});
        std::sort(ins.begin(), ins.end());
        const int uniq = (int)(std::unique(ins.begin(), ins.end()) - ins.begin());
        prof_begin(plan, 0, pass_bytes(pp.dev, L->n_nodes, uniq, !compact), st, &e1);
        if (compact && co->count)
          plan.prof.units.push_back({0, co->count, (double)L->n_nodes * (8.0 * (double)(1u << co->ctl))});
      }
      if (pp.jit_id >= 0) launch_pass_jit(*L, tiles, plan.jit_entries[pp.jit_id], st);
      else launch_pass(*L, tiles, plan.fuse_bits, plan.tile_bits, st);
      if (prof) prof_end(plan, e1, st);
    }
  }
}

}  // namespace

double segment_bytes(const SegmentPlan& s) {
  double b = 0;
  for (auto& pp : s.passes) b += pass_bytes(pp.dev, 1, 1);
  return b;
}

namespace {

// The union of the requests' selected ranges (sorted, disjoint, merged).
std::vector<Range> union_ranges(const std::vector<ExecReq>& reqs) {
  std::vector<Range> all;
  for (auto& r : reqs)
    if (r.n > 0) all.insert(all.end(), r.rs.begin(), r.rs.end());
  std::sort(all.begin(), all.end(), [](const Range& x, const Range& y) { return x.lo < y.lo; });
  std::vector<Range> out;
  for (auto& r : all) {
    if (r.hi <= r.lo) continue;
    if (!out.empty() && r.lo <= out.back().hi) out.back().hi = std::max(out.back().hi, r.hi);
    else out.push_back(r);
  }
  return out;
}

int64_t total_bits(const std::vector<ExecReq>& reqs) {
  int64_t t = 0;
  for (auto& r : reqs)
    if (!r.rs.empty()) t += r.n;
  return t;
}

size_t comp_bytes(const Plan& p, const std::vector<ExecReq>& reqs) {
  if (p.opts.precision != SF_PREC_COMPENSATED) return 0;
  size_t b = 0;
  for (auto& r : reqs)
    if (r.n > 0 && !r.rs.empty()) b += align256((size_t)r.n * 16);
  return b;
}

// Finals of one request in path order: final id and its selected leaves.
struct FinalCursor {
  const std::vector<Range>* rs = nullptr;
  int fb = 0;
  size_t ri = 0;
  uint64_t cur = 0;
  bool has = false;
  Final f{};
  void start(const std::vector<Range>& r, int fbits) {
    rs = &r;
    fb = fbits;
    ri = 0;
    cur = r.empty() ? 0 : (r[0].lo >> fb);
    advance();
  }
  void advance() {
    has = false;
    while (ri < rs->size()) {
      const uint64_t lo = (*rs)[ri].lo, hi = (*rs)[ri].hi;
      const uint64_t a = lo >> fb, b = (hi - 1) >> fb;
      if (cur < a) cur = a;
      if (cur > b) {
        ri++;
        continue;
      }
      f.fid = cur;
      f.all = true;
      std::memset(f.mask, 0, sizeof(f.mask));
      if (fb > 0) {
        const uint64_t glo = cur << fb, ghi = (cur + 1) << fb;
        uint64_t cnt = 0;
        // leaves of this final from every range that touches it
        for (size_t r2 = ri; r2 < rs->size() && (*rs)[r2].lo < ghi; r2++) {
          uint64_t l = std::max((*rs)[r2].lo, glo), h = std::min((*rs)[r2].hi, ghi);
          for (uint64_t v = l; v < h; v++) {
            uint64_t b2 = v - glo;
            f.mask[b2 >> 6] |= 1ull << (b2 & 63);
            cnt++;
          }
        }
        f.all = cnt == (1ull << fb);
      }
      cur++;
      has = true;
      return;
    }
  }
};

}  // namespace

size_t exec_workspace_bytes(const Plan& p, const std::vector<ExecReq>& reqs, int64_t budget) {
  const std::vector<Range> u = union_ranges(reqs);
  Layout lay = make_layout(p, count_finals(p, u), compact_plan(p, total_bits(reqs)), budget, comp_bytes(p, reqs));
  return lay.bytes + 256;
}

// Allocate a workspace for these requests. The plan's layout takes as many
// finals per launch as its memory budget allows; when the device has less
// free memory than that budget assumed (other allocations since the plan was
// made), the layout's budget is halved - fewer finals per launch - until the
// allocation succeeds, or fails with SF_ENOMEM once one final per block does
// not fit. Returns the budget the layout used (0: the plan's own), which the
// caller passes to exec_run (ExecCtx::budget).
int64_t exec_alloc_workspace(const Plan& p, const std::vector<ExecReq>& reqs, int64_t budget, void** ws,
                             size_t* bytes) {
  size_t need = exec_workspace_bytes(p, reqs, budget);
  while (true) {
    const cudaError_t e = cudaMalloc(ws, need);
    if (e == cudaSuccess) {
      *bytes = need;
      return budget;
    }
    if (e != cudaErrorMemoryAllocation) fail(SF_ECUDA, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
    cudaGetLastError();
    const int64_t next = (int64_t)((need - 256) / 2);
    size_t need2 = 0;
    try {
      need2 = exec_workspace_bytes(p, reqs, next);
    } catch (const Error&) {
      fail(SF_ENOMEM, "cudaMalloc workspace: out of memory (" + std::to_string(need) + " bytes)");
    }
    if (need2 >= need) fail(SF_ENOMEM, "cudaMalloc workspace: out of memory (" + std::to_string(need) + " bytes)");
    budget = next;
    need = need2;
  }
}

size_t exec_workspace_bytes(const Plan& p, int64_t n, const sf_path_sel& s, int64_t budget) {
  std::vector<ExecReq> one(1);
  double fa;
  one[0].rs = select_ranges(p, s, &fa);
  one[0].n = n;
  return exec_workspace_bytes(p, one, budget);
}

void prof_begin(Plan& p, int kind, double bytes, void* stream, void** e1_out, int launches) {
  p.prof.launches[kind] += launches;
  p.prof.bytes[kind] += bytes;
  *e1_out = nullptr;
  if (!p.prof.timing) return;
  cudaEvent_t e[2];
  for (int i = 0; i < 2; i++) {
    if (!p.prof.pool.empty()) {
      e[i] = (cudaEvent_t)p.prof.pool.back();
      p.prof.pool.pop_back();
    } else if (cudaEventCreate(&e[i]) != cudaSuccess) {
      fail(SF_ECUDA, "cudaEventCreate failed");
    }
  }
  cudaEventRecord(e[0], (cudaStream_t)stream);
  p.prof.pending.push_back({kind, (void*)e[0], (void*)e[1]});
  *e1_out = (void*)e[1];
}

void prof_end(Plan&, void* e1, void* stream) {
  if (e1) cudaEventRecord((cudaEvent_t)e1, (cudaStream_t)stream);
}

void prof_collect(Plan& p) {
  for (auto& r : p.prof.pending) {
    cudaEventSynchronize((cudaEvent_t)r.e1);
    float ms = 0;
    if (cudaEventElapsedTime(&ms, (cudaEvent_t)r.e0, (cudaEvent_t)r.e1) == cudaSuccess)
      p.prof.seconds[r.kind] += ms * 1e-3;
    p.prof.pool.push_back(r.e0);
    p.prof.pool.push_back(r.e1);
  }
  p.prof.pending.clear();
  // the counters are written by kernels on the callers' streams
  if (!p.prof.units.empty()) cudaDeviceSynchronize();
  for (auto& u : p.prof.units) {
    uint32_t v = 0;
    if (cudaMemcpy(&v, u.count, sizeof(v), cudaMemcpyDeviceToHost) == cudaSuccess) p.prof.bytes[u.kind] += v * u.unit;
  }
  p.prof.units.clear();
}

void prof_release(Plan& p) {
  prof_collect(p);
  for (void* e : p.prof.pool) cudaEventDestroy((cudaEvent_t)e);
  p.prof.pool.clear();
}

namespace {
// The last cache (identified by its slot) that ran in each workspace: a
// cache may reuse the nodes it left in a workspace only if no other plan or
// caller context ran there since.
std::mutex g_ws_mu;
std::unordered_map<const void*, const void*> g_ws_owner;
}  // namespace

void exec_forget_workspace(const void* ws) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  g_ws_owner.erase(ws);
}

void exec_release_cache(Plan& p) {
  delete reinterpret_cast<Cache*>(p.cache);
  p.cache = nullptr;
}

void exec_free_cache(void* c) { delete reinterpret_cast<Cache*>(c); }

void exec_run(Plan& plan, const uint64_t* d_bits, int64_t n, const sf_path_sel& sel, double* d_out,
              int accumulate, void* ws, size_t ws_bytes, void* stream, bool keep_cache, ExecCtx* ctx) {
  if (n < 0) fail(SF_EINVAL, "negative bitstring count");
  std::vector<ExecReq> one(1);
  double fa = 0;
  one[0].rs = select_ranges(plan, sel, &fa);
  one[0].d_bits = d_bits;
  one[0].n = n;
  one[0].d_out = d_out;
  one[0].accumulate = accumulate;
  one[0].cancel = ctx ? ctx->cancel : nullptr;
  exec_run(plan, one, ws, ws_bytes, stream, keep_cache, ctx);
}

void exec_run(Plan& plan, std::vector<ExecReq>& reqs, void* ws, size_t ws_bytes, void* stream, bool keep_cache,
              ExecCtx* ctx) {
  cudaStream_t st = (cudaStream_t)stream;
  void** cache_slot = (ctx && ctx->cache_slot) ? ctx->cache_slot : &plan.cache;
  const bool prof = ctx ? ctx->profile : true;
  int* err = (ctx && ctx->err) ? ctx->err : plan.d_err;
  const uint32_t* tabA = plan.d_tabA;
  const uint32_t* tabB = plan.d_tabB;
  const int64_t budget = ctx ? ctx->budget : 0;
  const bool compensated = plan.opts.precision == SF_PREC_COMPENSATED;
  for (auto& r : reqs) {
    if (r.n < 0) fail(SF_EINVAL, "negative bitstring count");
    r.cancelled = false;
    if (r.n > 0 && !r.accumulate) {
      void* e1 = nullptr;
      if (prof) prof_begin(plan, 2, 16.0 * r.n, st, &e1);
      launch_zero(r.d_out, 2 * r.n, st);
      if (prof) prof_end(plan, e1, st);
    }
  }
  const std::vector<Range> urs = union_ranges(reqs);
  const int64_t ntot = total_bits(reqs);
  if (ntot == 0 || urs.empty()) return;
  if (!tabA || !tabB || !err) fail(SF_EINVAL, "internal: plan has no device state");
  const uint64_t nfin = count_finals(plan, urs);
  const Compact cp = compact_plan(plan, ntot);
  const size_t cb = comp_bytes(plan, reqs);
  Layout lay = make_layout(plan, nfin, cp, budget, cb);
  const size_t nb = node_bytes(plan);
  const size_t need = lay.bytes + 256;
  if (!ws || ws_bytes < need)
    fail(SF_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes");
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~(uintptr_t)255);

  Cache* C = reinterpret_cast<Cache*>(*cache_slot);
  bool same_owner;
  {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto it = g_ws_owner.find(ws);
    same_owner = it != g_ws_owner.end() && it->second == (const void*)cache_slot;
    g_ws_owner[ws] = (const void*)cache_slot;
  }
  if (!C || !keep_cache || !same_owner || C->ws != ws || C->ws_bytes != ws_bytes || C->B != lay.B ||
      C->cap != lay.cap) {
    delete C;
    C = new Cache();
    *cache_slot = C;
    C->ws = ws;
    C->ws_bytes = ws_bytes;
    C->B = lay.B;
    C->cap = lay.cap;
    size_t at = 0;
    for (size_t s = 0; s < lay.cap.size(); s++) {
      C->first_slot.push_back(at);
      C->slots.emplace_back(lay.cap[s]);
      at += lay.cap[s];
    }
    C->final_first = at;
  }
  const int nL = (int)plan.levels.size();
  const size_t bytesA = ((size_t)1 << plan.A.m) * 8;
  auto bufA = [&](size_t slot) { return (void*)(base + slot * nb); };
  auto bufB = [&](size_t slot) { return (void*)(base + slot * nb + bytesA); };
  const int fb = plan.deferred ? plan.defer_bits : 0;
  // nc cached depths 0 .. nc-1; a final's parent is its node at depth nc-1,
  // sh_f path bits (of the final id) above it
  const int nc = cached_depths(plan);
  int sh_f = 0;
  if (plan.merged_last) sh_f = nL >= 2 ? plan.levels[nL - 2].bits : 0;
  else if (!plan.deferred) sh_f = nL > 0 ? plan.levels[nL - 1].bits : 0;
  const SegmentPlan& finA =
      plan.merged_last ? plan.A.last_merged : (plan.deferred ? plan.A.last_deferred : plan.A.seg[nL]);
  const SegmentPlan& finB =
      plan.merged_last ? plan.B.last_merged : (plan.deferred ? plan.B.last_deferred : plan.B.seg[nL]);

  // the pass kernels' work counters (the last bytes), zeroed once per call
  uint32_t* work = reinterpret_cast<uint32_t*>(base + (lay.bytes - kWorkBytes));
  launch_zero(reinterpret_cast<double*>(work), 1, st);
  // compensation terms of each request (after everything else), zeroed
  char* comp_at = base + (lay.bytes - kWorkBytes - cb);
  std::vector<double*> comp(reqs.size(), nullptr);
  if (compensated)
    for (size_t q = 0; q < reqs.size(); q++) {
      if (reqs[q].n <= 0 || reqs[q].rs.empty()) continue;
      comp[q] = reinterpret_cast<double*>(comp_at);
      comp_at += align256((size_t)reqs[q].n * 16);
      launch_zero(comp[q], 2 * reqs[q].n, st);
    }

  // compact finals: block maps after the node slots, then B finals' buffers;
  // the maps are built once per call from every request's bitstrings
  uint32_t* cmap[2] = {nullptr, nullptr};
  char* cfin = nullptr;
  const uint32_t* ccount[2] = {nullptr, nullptr};
  if (lay.compact) {
    char* at = base + align256(lay.total_slots * nb);
    BlockMapLaunch M;
    std::memset(&M, 0, sizeof(M));
    M.tab[0] = tabA;
    M.tab[1] = tabB;
    uint32_t* cnt = nullptr;
    if (prof && plan.d_cnt) {
      if (plan.cnt_seq > 0 && plan.cnt_seq % kCountRing == 0) prof_collect(plan);
      cnt = plan.d_cnt + 2 * (plan.cnt_seq % kCountRing);
      plan.cnt_seq++;
    }
    double mb = 8.0 * (double)ntot;
    int nk = 2;
    for (int side = 0; side < 2; side++) {
      if (!cp.s[side].on) continue;
      cmap[side] = reinterpret_cast<uint32_t*>(at);
      at += cp.s[side].map_bytes;
      M.map[side] = cmap[side];
      M.c[side] = cp.s[side].c;
      M.nw[side] = (int64_t)cp.s[side].nw;
      M.sums[side] = reinterpret_cast<uint32_t*>(at);
      at += cp.s[side].sums_bytes;
      M.count[side] = cnt ? cnt + side : nullptr;
      ccount[side] = M.count[side];
      mb += 28.0 * (double)cp.s[side].nw;  // zero, count, rank
      nk++;
    }
    cfin = at;
    std::vector<std::pair<const uint64_t*, int64_t>> sets;
    for (auto& r : reqs)
      if (r.n > 0 && !r.rs.empty()) {
        sets.push_back({r.d_bits, r.n});
        nk++;
      }
    void* e1 = nullptr;
    if (prof) prof_begin(plan, 2, mb, st, &e1, nk);
    launch_block_maps(M, sets, st);
    if (prof) prof_end(plan, e1, st);
  }
  auto cbuf = [&](size_t i, int side) -> void* {
    return cfin + i * cp.per_final + (side && cp.s[0].on ? cp.s[0].buf_bytes : 0);
  };

  // gather template (per request: bits, n, acc, comp)
  GatherLaunch G;
  std::memset(&G, 0, sizeof(G));
  G.tabA = tabA;
  G.tabB = tabB;
  G.g = plan.deferred ? plan.levels.back().n_cross : 0;
  G.nterm_bits = plan.deferred ? plan.cross[plan.levels.back().first_cross].bits : 0;
  for (int side = 0; side < 2; side++) {
    const SegmentPlan& fin = side ? finB : finA;
    const HalfPlan& H = side ? plan.B : plan.A;
    GatherSide& gs = side ? G.B : G.A;
    if (cmap[side]) {
      gs.c = cp.s[side].c;
      gs.c.cmap = cmap[side];
    }
    if (fin.pins_out.size() > (size_t)MAX_PINS) fail(SF_EUNSUPPORTED, "too many pins at gather");
    gs.npin = (int)fin.pins_out.size();
    for (size_t i = 0; i < fin.pins_out.size(); i++) {
      const Pin& pn = fin.pins_out[i];
      gs.pin[i].pos = (int8_t)pn.pos;
      gs.pin[i].xi = (int8_t)pn.xi;
      for (int t = 0; t < 4; t++) gs.pin[i].v[t] = (uint8_t)pn.v[t];
    }
    for (int t = 0; t < G.g; t++) {
      const CrossGate& x = plan.cross[plan.levels.back().first_cross + t];
      int q = side ? x.qb : x.qa;
      gs.dpos[t] = (int8_t)H.pos_of[q];
      gs.dq[t] = (int8_t)q;
    }
  }
  std::memcpy(G.ma, plan.ma, sizeof(G.ma));
  std::memcpy(G.mb, plan.mb, sizeof(G.mb));
  for (size_t i = 0; i < plan.cross.size(); i++) {
    G.xshift[i] = (uint8_t)plan.cross[i].shift;
    G.xbits[i] = (uint8_t)plan.cross[i].bits;
  }

  // finals of the union in path order; per final, the requests that select
  // leaves of it (and which)
  std::vector<FinalCursor> cur(reqs.size());
  for (size_t q = 0; q < reqs.size(); q++) {
    if (reqs[q].n > 0) cur[q].start(reqs[q].rs, fb);
  }
  struct UFinal {
    uint64_t fid;
    std::vector<std::pair<int, Final>> who;
  };
  auto next_final = [&](UFinal& u) -> bool {
    uint64_t best = ~0ull;
    for (auto& c : cur)
      if (c.rs && c.has) best = std::min(best, c.f.fid);
    if (best == ~0ull) return false;
    u.fid = best;
    u.who.clear();
    for (size_t q = 0; q < cur.size(); q++)
      if (cur[q].rs && cur[q].has && cur[q].f.fid == best) {
        u.who.push_back({(int)q, cur[q].f});
        cur[q].advance();
      }
    return true;
  };

  std::vector<UFinal> block;
  std::vector<std::vector<GatherFinal>> gf(reqs.size());
  try {
    UFinal f;
    bool more = next_final(f);
    while (more) {
      int live = 0;
      for (auto& r : reqs) {
        if (r.cancel && *r.cancel) r.cancelled = true;
        if (r.n > 0 && !r.rs.empty() && !r.cancelled) live++;
      }
      if (live == 0) fail(SF_ECANCELLED, "request cancelled");
      block.clear();
      while (more && (int)block.size() < lay.B) {
        block.push_back(f);
        more = next_final(f);
      }
      // parents at depth nc-1 (ids) of the block's finals
      std::vector<uint64_t> pid(block.size());
      for (size_t i = 0; i < block.size(); i++) pid[i] = block[i].fid >> sh_f;
      // cached depths 0 .. nc-1
      std::vector<int> prev_slot;  // slot index (within depth) per needed node at depth s-1
      std::vector<uint64_t> prev_ids;
      for (int s = 0; s < nc; s++) {
        const int below = total_bits_below(plan, s) - (nc > 0 ? total_bits_below(plan, nc - 1) : 0);
        // node id at depth s = pid >> (bits of levels s .. nc-2)
        std::vector<uint64_t> ids;
        for (uint64_t v : pid) {
          uint64_t id = below >= 64 ? 0 : (v >> below);
          if (ids.empty() || ids.back() != id) ids.push_back(id);
        }
        auto& slots = C->slots[s];
        std::vector<int> where(ids.size(), -1);
        std::vector<bool> keep(slots.size(), false);
        {
          std::unordered_map<uint64_t, int> resident;
          for (size_t q = 0; q < slots.size(); q++)
            if (slots[q].valid) resident[slots[q].id] = (int)q;
          for (size_t i = 0; i < ids.size(); i++) {
            auto it = resident.find(ids[i]);
            if (it != resident.end()) {
              where[i] = it->second;
              keep[it->second] = true;
            }
          }
        }
        size_t freep = 0;
        std::vector<Job> jobsA, jobsB;
        std::vector<size_t> computed;
        for (size_t i = 0; i < ids.size(); i++) {
          if (where[i] >= 0) continue;
          while (freep < slots.size() && keep[freep]) freep++;
          if (freep >= slots.size()) fail(SF_EINVAL, "internal: slot capacity");
          where[i] = (int)freep;
          keep[freep] = true;
          Slot& sl = slots[freep];
          sl.id = ids[i];
          sl.valid = false;
          const uint64_t path = (total_bits_below(plan, s) >= 64) ? 0 : (ids[i] << total_bits_below(plan, s));
          // parent
          const void *inA = nullptr, *inB = nullptr;
          bool pdead = false;
          cd psa = plan.A.root_scale, psb = plan.B.root_scale;
          if (s > 0) {
            const uint64_t parent = ids[i] >> plan.levels[s - 1].bits;
            size_t pi = std::lower_bound(prev_ids.begin(), prev_ids.end(), parent) - prev_ids.begin();
            if (pi >= prev_ids.size() || prev_ids[pi] != parent) fail(SF_EINVAL, "internal: parent missing");
            const Slot& ps = C->slots[s - 1][prev_slot[pi]];
            pdead = ps.dead;
            psa = ps.sa;
            psb = ps.sb;
            inA = bufA(C->first_slot[s - 1] + prev_slot[pi]);
            inB = bufB(C->first_slot[s - 1] + prev_slot[pi]);
          }
          const SegmentPlan& sA = plan.A.seg[s];
          const SegmentPlan& sB = plan.B.seg[s];
          sl.dead = pdead || dead_by_pins(sA.passes[0].dev, plan, path) || dead_by_pins(sB.passes[0].dev, plan, path);
          sl.sa = psa * sA.scale;
          sl.sb = psb * sB.scale;
          if (!sl.dead) {
            jobsA.push_back({inA, bufA(C->first_slot[s] + freep), path});
            jobsB.push_back({inB, bufB(C->first_slot[s] + freep), path});
          }
          computed.push_back(freep);
        }
        run_segment(*C, plan, plan.A.seg[s], jobsA, st, prof, err, work);
        run_segment(*C, plan, plan.B.seg[s], jobsB, st, prof, err, work);
        for (size_t q : computed) slots[q].valid = true;
        prev_ids = ids;
        prev_slot = where;
      }
      // finals
      std::vector<Job> jobsA, jobsB;
      for (auto& v : gf) v.clear();
      CompactOut coA, coB;
      for (int side = 0; side < 2; side++) {
        CompactOut& co = side ? coB : coA;
        co.cmap = cmap[side];
        co.ctl = cp.s[side].c.ctl;
        co.count = ccount[side];
      }
      for (size_t i = 0; i < block.size(); i++) {
        const uint64_t fpath = block[i].fid << fb;
        const void *inA = nullptr, *inB = nullptr;
        bool pdead = false;
        cd psa = plan.A.root_scale, psb = plan.B.root_scale;
        if (nc > 0) {
          size_t pi = std::lower_bound(prev_ids.begin(), prev_ids.end(), pid[i]) - prev_ids.begin();
          if (pi >= prev_ids.size() || prev_ids[pi] != pid[i]) fail(SF_EINVAL, "internal: final parent missing");
          const Slot& ps = C->slots[nc - 1][prev_slot[pi]];
          pdead = ps.dead;
          psa = ps.sa;
          psb = ps.sb;
          inA = bufA(C->first_slot[nc - 1] + prev_slot[pi]);
          inB = bufB(C->first_slot[nc - 1] + prev_slot[pi]);
        }
        bool dead = pdead || dead_by_pins(finA.passes[0].dev, plan, fpath) ||
                    dead_by_pins(finB.passes[0].dev, plan, fpath);
        bool wanted = false;  // by a request that is still live
        for (auto& w : block[i].who)
          if (!reqs[w.first].cancelled) wanted = true;
        if (dead || !wanted) continue;
        const size_t fs = C->final_first + i;
        jobsA.push_back({inA, bufA(fs), fpath});
        jobsB.push_back({inB, bufB(fs), fpath});
        GatherFinal g;
        std::memset(&g, 0, sizeof(g));
        g.wa = bufA(fs);
        g.wb = bufB(fs);
        if (cmap[0]) {
          coA.out.push_back(cbuf(i, 0));
          g.wa = coA.out.back();
        }
        if (cmap[1]) {
          coB.out.push_back(cbuf(i, 1));
          g.wb = coB.out.back();
        }
        g.path = fpath;
        cd sc = psa * finA.scale * psb * finB.scale;
        g.sre = sc.real();
        g.sim = sc.imag();
        for (auto& w : block[i].who) {
          if (reqs[w.first].cancelled) continue;
          g.all_leaves = w.second.all ? 1 : 0;
          std::memcpy(g.leafmask, w.second.mask, sizeof(g.leafmask));
          gf[w.first].push_back(g);
        }
      }
      run_segment(*C, plan, finA, jobsA, st, prof, err, work, cmap[0] ? &coA : nullptr);
      run_segment(*C, plan, finB, jobsB, st, prof, err, work, cmap[1] ? &coB : nullptr);
      if (plan.opts.exec_mode == SF_EXEC_PLAIN) {
        // the plain form shares nothing below the selection prefix: every
        // path re-evolves its levels under the prefix checkpoint
        int cum = 0;
        for (int s = 0; s < nc; s++) {
          if (cum > plan.xs)
            for (auto& sl : C->slots[s]) sl.valid = false;
          cum += plan.levels[s].bits;
        }
      }
      for (size_t q = 0; q < reqs.size(); q++) {
        const ExecReq& r = reqs[q];
        if (gf[q].empty() || r.cancelled) continue;
        G.bits = r.d_bits;
        G.n = r.n;
        G.acc = r.d_out;
        G.comp = comp[q];
        for (size_t g0 = 0; g0 < gf[q].size(); g0 += GATHER_FINALS) {
          size_t g1 = std::min(gf[q].size(), g0 + GATHER_FINALS);
          G.n_finals = (int)(g1 - g0);
          for (size_t j = g0; j < g1; j++) G.finals[j - g0] = gf[q][j];
          void* e1 = nullptr;
          const double gb = (double)r.n * (8.0 + 32.0 + 16.0 * G.n_finals * (2 << G.g));
          if (prof) prof_begin(plan, 1, gb, st, &e1);
          launch_gather(G, st);
          if (prof) prof_end(plan, e1, st);
        }
      }
    }
    if (compensated)
      for (size_t q = 0; q < reqs.size(); q++)
        if (comp[q] && !reqs[q].cancelled) {
          void* e1 = nullptr;
          if (prof) prof_begin(plan, 2, 48.0 * reqs[q].n, st, &e1);
          launch_fold(reqs[q].d_out, comp[q], 2 * reqs[q].n, st);
          if (prof) prof_end(plan, e1, st);
        }
  } catch (...) {
    for (auto& v : C->slots)
      for (auto& sl : v) sl.valid = false;
    throw;
  }
  if (!keep_cache) {
    for (auto& v : C->slots)
      for (auto& sl : v) sl.valid = false;
  }
}

}  // namespace sf
