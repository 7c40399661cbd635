// Device code shared by the library's generic pass kernel and the run-time
// specialised pass kernels (compiled from this text by NVRTC): register-block
// gate bodies, mbarrier and copy helpers, and the warp-specialised pass body,
// a template over the stage program that the compute warps run on each tile.
#pragma once

#include "dev_types.h"

namespace sf {

__device__ __forceinline__ int digit_of(const uint8_t* xshift, const uint8_t* xbits, uint64_t path,
                                        int xi) {
  return (int)((path >> xshift[xi]) & ((1u << xbits[xi]) - 1u));
}

// count of trailing zeros, folded at compile time for unrolled loop indices
__host__ __device__ constexpr int cctz(int v) {
  int r = 0;
  while (v && !(v & 1)) {
    v >>= 1;
    r++;
  }
  return r;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// ---- register-block gate kernels (J = register bit, compile time) --------
template <int R, int J>
__device__ __forceinline__ void g_h(float2* v) {
#pragma unroll
  for (int i = 0; i < (1 << R); i++) {
    if (i & (1 << J)) continue;
    float2 a = v[i], b = v[i | (1 << J)];
    v[i] = make_float2(a.x + b.x, a.y + b.y);
    v[i | (1 << J)] = make_float2(a.x - b.x, a.y - b.y);
  }
}
// X^1/2 = (e^{i pi/4}/sqrt2) [[1, -i], [-i, 1]]: out0 = a - i b, out1 = b - i a
template <int R, int J>
__device__ __forceinline__ void g_xh(float2* v) {
#pragma unroll
  for (int i = 0; i < (1 << R); i++) {
    if (i & (1 << J)) continue;
    float2 a = v[i], b = v[i | (1 << J)];
    v[i] = make_float2(a.x + b.y, a.y - b.x);
    v[i | (1 << J)] = make_float2(b.x + a.y, b.y - a.x);
  }
}
// Y^1/2 = (e^{i pi/4}/sqrt2) [[1, -1], [1, 1]]: out0 = a - b, out1 = a + b
template <int R, int J>
__device__ __forceinline__ void g_yh(float2* v) {
#pragma unroll
  for (int i = 0; i < (1 << R); i++) {
    if (i & (1 << J)) continue;
    float2 a = v[i], b = v[i | (1 << J)];
    v[i] = make_float2(a.x - b.x, a.y - b.y);
    v[i | (1 << J)] = make_float2(a.x + b.x, a.y + b.y);
  }
}
template <int R, int J>
__device__ __forceinline__ void g_1(float2* v, float2 m0, float2 m1, float2 m2, float2 m3) {
#pragma unroll
  for (int i = 0; i < (1 << R); i++) {
    if (i & (1 << J)) continue;
    float2 a = v[i], b = v[i | (1 << J)];
    v[i] = cadd(cmul(m0, a), cmul(m1, b));
    v[i | (1 << J)] = cadd(cmul(m2, a), cmul(m3, b));
  }
}
template <int R, int J>
__device__ __forceinline__ void g_dmul(float2* v, float2 f0, float2 f1) {
#pragma unroll
  for (int i = 0; i < (1 << R); i++) v[i] = cmul((i & (1 << J)) ? f1 : f0, v[i]);
}
// 4x4 on register bits (A = high basis bit, B = low basis bit)
template <int R, int A, int B>
__device__ __forceinline__ void g_2(float2* v, const float* m) {
#pragma unroll
  for (int i = 0; i < (1 << R); i++) {
    if (i & ((1 << A) | (1 << B))) continue;
    const int i0 = i, i1 = i | (1 << B), i2 = i | (1 << A), i3 = i | (1 << A) | (1 << B);
    float2 x[4] = {v[i0], v[i1], v[i2], v[i3]};
    float2 y[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        float2 mm = make_float2(m[2 * (4 * r + c)], m[2 * (4 * r + c) + 1]);
        acc = cadd(acc, cmul(mm, x[c]));
      }
      y[r] = acc;
    }
    v[i0] = y[0];
    v[i1] = y[1];
    v[i2] = y[2];
    v[i3] = y[3];
  }
}

// a * e^{i pi K/4} for a compile-time K (h = 1/sqrt2 rounded to float)
template <int K>
__device__ __forceinline__ float2 omega_mul(float2 a) {
  constexpr float h = 0.70710678118654752f;
  if constexpr (K == 0) return a;
  else if constexpr (K == 1) return make_float2((a.x - a.y) * h, (a.x + a.y) * h);
  else if constexpr (K == 2) return make_float2(-a.y, a.x);
  else if constexpr (K == 3) return make_float2(-(a.x + a.y) * h, (a.x - a.y) * h);
  else if constexpr (K == 4) return make_float2(-a.x, -a.y);
  else if constexpr (K == 5) return make_float2((a.y - a.x) * h, -(a.x + a.y) * h);
  else if constexpr (K == 6) return make_float2(a.y, -a.x);
  else return make_float2((a.x + a.y) * h, (a.y - a.x) * h);
}

__device__ __forceinline__ uint32_t pin_val(const DevPin& p, const uint8_t* xshift, const uint8_t* xbits,
                                            uint64_t path) {
  return p.xi < 0 ? p.v[0] : p.v[digit_of(xshift, xbits, path, p.xi)];
}

// ---- mbarriers and asynchronous copies (inline PTX) ------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Wait for phase `parity` of the barrier, giving up after ~2^31 cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

// Per-item geometry: tile base index and pin masks (tile-local and run-level).
struct ItemGeo {
  uint32_t base;                 // global index bits of the tile (inactive bits)
  uint32_t lin_m, lin_v;         // input pins on tile-local bits
  uint32_t lout_m, lout_v;       // output pins on tile-local bits
  uint32_t tile;                 // tile number (the free positions of base, packed)
  int node;
  uint64_t path;
};

__device__ __forceinline__ ItemGeo item_geo(const PassLaunch& P, int64_t item, int tiles_log2) {
  const DevPass& d = P.pass;
  ItemGeo g;
  // tile-major order: the launch's nodes take tile t one after another, so
  // nodes that read one parent buffer (siblings) fetch each of its tiles from
  // DRAM once and from L2 after that
  g.node = (int)(item % P.n_nodes);
  const uint32_t t = (uint32_t)(item / P.n_nodes);
  g.tile = t;
  g.path = P.nodes[g.node].path;
  uint32_t base = 0;
  for (int i = 0; i < d.n_free; i++) base |= ((t >> i) & 1u) << d.freepos[i];
  uint32_t active = 0;
  for (int j = 0; j < d.k; j++) active |= 1u << d.gpos[j];
  uint32_t pm = 0, pv = 0, om = 0, ov = 0;
  for (int i = 0; i < d.n_pin_in; i++) {
    const uint32_t b = 1u << d.pin_in[i].pos;
    pm |= b;
    if (pin_val(d.pin_in[i], P.xshift, P.xbits, g.path)) pv |= b;
  }
  for (int i = 0; i < d.n_pin_out; i++) {
    const uint32_t b = 1u << d.pin_out[i].pos;
    om |= b;
    if (pin_val(d.pin_out[i], P.xshift, P.xbits, g.path)) ov |= b;
  }
  g.base = base | (pv & ~active);
  g.lin_m = g.lin_v = g.lout_m = g.lout_v = 0;
  for (int j = 0; j < d.k; j++) {
    const uint32_t gb = 1u << d.gpos[j];
    if (pm & gb) {
      g.lin_m |= 1u << j;
      if (pv & gb) g.lin_v |= 1u << j;
    }
    if (om & gb) {
      g.lout_m |= 1u << j;
      if (ov & gb) g.lout_v |= 1u << j;
    }
  }
  return g;
}

__device__ __forceinline__ void compute_bar(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
__device__ __forceinline__ bool compute_bar_or(int nthreads, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(nthreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// 16 zero bytes at a shared-memory address (a chunk of a pinned-out run)
__device__ __forceinline__ void st_shared_zero16(uint32_t dst) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0u) : "memory");
}
// the barrier's pending count drops by one when this thread's earlier
// cp.async copies have landed
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Persistent fused pass, warp-specialised. Each CTA walks work items
// (node, tile) with stride gridDim.x through NBUF shared-memory tile buffers.
// Warp roles: compute warps run the register stages; a load warp streams the
// next tiles in with 16-byte cp.async copies (one warp instruction moves 512
// contiguous-run bytes; completion arrives on full[b]); a store warp streams
// finished tiles out with 16-byte vector stores once the compute warps arrive
// on empty[b], then frees the buffer (free[b]). Input-pinned (structurally
// zero) runs are never read and output-pinned runs never written. Every wait
// is bounded; a timeout sets the error flag and ends the kernel.
// Copy geometry of a tile: run r (2^L contiguous amplitudes) of a tile sits
// at global offset runoff[r]; chunk c (elements 2c, 2c+1) at swz(2c). The
// load warp writes zeros for the chunks of input-pinned runs (structural
// zeros, never read); the compute warps zero the elements pinned out inside
// a run.
struct CopyCtx {
  const uint32_t* runoff;
  int L, nchunk;
  uint32_t lmask;
};

// The generic copy loops: four 16-byte chunks in flight per lane. They use
// the default tile swizzle; a stage program with its own swizzle defines
// swz() and its own copies.
struct GenericCopy {
  static __device__ __forceinline__ uint32_t swz(uint32_t e) { return sf::swz(e); }
  static __device__ __forceinline__ ItemGeo geo(const PassLaunch& P, int64_t item, int tiles_log2) {
    return item_geo(P, item, tiles_log2);
  }
  static __device__ __forceinline__ void load_tile(const PassLaunch& P, const ItemGeo& g, uint32_t dst, int lane,
                                                   const CopyCtx& cc) {
    const float2* in = reinterpret_cast<const float2*>(P.nodes[g.node].in);
    const uint32_t rm = g.lin_m >> cc.L, rv = g.lin_v >> cc.L;
    for (int c0 = lane; c0 < cc.nchunk; c0 += 128) {
      uint32_t so[4];
      const float2* src[4];
      bool ok[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int c = c0 + 32 * u;
        const int e = c << 1, r = e >> cc.L;
        ok[u] = c < cc.nchunk && (((uint32_t)r & rm) == rv);
        so[u] = swz((uint32_t)e) * 8u;
        src[u] = in + (g.base | cc.runoff[ok[u] ? r : 0] | (uint32_t)(e & cc.lmask));
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (ok[u]) cp_async16(dst + so[u], src[u]);
        else if (c0 + 32 * u < cc.nchunk) st_shared_zero16(dst + so[u]);  // pinned-out run
      }
    }
  }
  static __device__ __forceinline__ void store_tile(const PassLaunch& P, const ItemGeo& g, const float2* buf,
                                                    int lane, const CopyCtx& cc) {
    float2* out = reinterpret_cast<float2*>(P.nodes[g.node].out);
    const float4* srcb = reinterpret_cast<const float4*>(buf);
    const uint32_t rm = g.lout_m >> cc.L, rv = g.lout_v >> cc.L;
    for (int c0 = lane; c0 < cc.nchunk; c0 += 128) {
      float4 v[4];
      float2* dst[4];
      bool ok[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int c = c0 + 32 * u;
        const int e = c << 1, r = e >> cc.L;
        ok[u] = c < cc.nchunk && (((uint32_t)r & rm) == rv);
        v[u] = srcb[swz((uint32_t)(ok[u] ? e : 0)) >> 1];
        dst[u] = out + (g.base | cc.runoff[ok[u] ? r : 0] | (uint32_t)(e & cc.lmask));
      }
#pragma unroll
      for (int u = 0; u < 4; u++)
        if (ok[u]) *reinterpret_cast<float4*>(dst[u]) = v[u];
    }
  }
};

// Compact store of a final pass (PassLaunch::cmap set): the tile's parts
// (2^ctl consecutive elements each, the tile's share of one block of the
// gather) are consecutive bits of the part map; a lane takes 32 of them per
// round, one 8-byte load of (map word, prefix count), and writes each
// requested part to its slot as 16-byte chunks. The store warp loads the
// first round's words as soon as the tile's geometry is published, while the
// compute warps work on the tile.
struct CompactWord {
  uint32_t bits;  // requested parts among the lane's 32 (bit j: part ub + j)
  uint32_t rank;  // requested parts of the half below part ub
};

__device__ __forceinline__ CompactWord compact_word(const PassLaunch& P, const ItemGeo& g, int lane, int r) {
  const int kt = P.pass.k - P.ctl;
  const uint32_t nparts = 1u << kt;
  const uint32_t ub = 32u * (uint32_t)(lane + 32 * r);
  CompactWord cw{0u, 0u};
  if (ub >= nparts) return cw;
  const uint64_t pb = ((uint64_t)g.tile << kt) + ub;  // part number of part ub
  const uint2 w = reinterpret_cast<const uint2*>(P.cmap)[pb >> 5];
  const uint32_t off = (uint32_t)pb & 31u;  // nonzero only for tiles of < 32 parts
  const uint32_t cnt = nparts - ub < 32u ? nparts - ub : 32u;
  cw.bits = (w.x >> off) & (cnt == 32u ? 0xffffffffu : ((1u << cnt) - 1u));
  cw.rank = w.y + (uint32_t)__popc(w.x & ((1u << off) - 1u));
  return cw;
}

// SW::swz is the tile's shared-memory swizzle.
template <class SW>
__device__ __forceinline__ void compact_write(const PassLaunch& P, const ItemGeo& g, const float2* buf, int lane,
                                              int r, const CompactWord& cw) {
  float2* out = reinterpret_cast<float2*>(P.nodes[g.node].out);
  const float4* srcb = reinterpret_cast<const float4*>(buf);
  const int tl = P.ctl;
  const int nq = 1 << (tl - 1);  // 16-byte chunks per part
  const uint32_t ub = 32u * (uint32_t)(lane + 32 * r);
  uint32_t bits = cw.bits;
  while (bits) {
    const uint32_t j = (uint32_t)__ffs(bits) - 1u;
    bits &= bits - 1u;
    const uint32_t slot = cw.rank + (uint32_t)__popc(cw.bits & ((1u << j) - 1u));
    float4* dst = reinterpret_cast<float4*>(out + ((uint64_t)slot << tl));
    const uint32_t c0 = (ub + j) << (tl - 1);
    for (int q = 0; q < nq; q++) dst[q] = srcb[SW::swz(2u * (c0 + (uint32_t)q)) >> 1];
  }
}

// cw: the lane's words of round 0 (compact_word(P, g, lane, 0)).
template <class SW>
__device__ __forceinline__ void compact_store_tile(const PassLaunch& P, const ItemGeo& g, const float2* buf,
                                                   int lane, const CompactWord& cw) {
  const int kt = P.pass.k - P.ctl;
  const int rounds = kt > 10 ? 1 << (kt - 10) : 1;
  compact_write<SW>(P, g, buf, lane, 0, cw);
  for (int r = 1; r < rounds; r++) compact_write<SW>(P, g, buf, lane, r, compact_word(P, g, lane, r));
}

// Prog::run(P, sm, g, w8, ncomp, active) runs the register stages of one
// tile: every compute thread calls it and passes each stage barrier at the
// same instruction; only active threads (below 2^(k-R)) do stage work.
// Prog::load_tile / Prog::store_tile move a tile between its node buffer and
// shared memory (load warp: cp.async into dst; store warp: vector stores).
// NBUF tile buffers (3: load, compute and store each on their own buffer;
// 2: half the shared memory, so that more CTAs fit on an SM).
template <int R, class Prog, int NBUF = 3>
__device__ __forceinline__ void pass_body(const PassLaunch& P) {
  extern __shared__ __align__(128) unsigned char smem[];
  const DevPass& d = P.pass;
  const int k = d.k, L = d.L;
  const int ntile = 1 << k, nruns = 1 << (k - L);
  const int nact = 1 << (k - R);                 // compute threads doing stage work
  const int ncw = (nact + 31) >> 5;               // compute warps
  const int ncomp = ncw * 32;
  float2* bufs = reinterpret_cast<float2*>(smem);
  uint32_t* runoff = reinterpret_cast<uint32_t*>(bufs + NBUF * ntile);
  uint64_t* full = reinterpret_cast<uint64_t*>(runoff + ((nruns + 1) & ~1));
  uint64_t* empty = full + NBUF;
  uint64_t* freeb = empty + NBUF;
  __shared__ float2 w8[8];
  __shared__ int abort_flag;
  __shared__ ItemGeo geo[NBUF];  // geometry of the item in buffer b
  const int tiles_log2 = d.n_free;
  const int64_t items = (int64_t)P.n_nodes << tiles_log2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = ntile >> 1;                  // 16-byte chunks per tile
  const int lmask = (1 << L) - 1;

  if (threadIdx.x < 8) {
    const float r = 0.70710678118654752f;
    const float c = (threadIdx.x & 1) ? r : 1.0f;
    const int t = threadIdx.x;
    float re = (t == 0) ? 1.f : (t == 2 || t == 6) ? 0.f : (t == 4) ? -1.f : (t == 1 || t == 7) ? c : -c;
    float im = (t == 2) ? 1.f : (t == 6) ? -1.f : (t == 0 || t == 4) ? 0.f : (t == 1 || t == 3) ? c : -c;
    w8[t] = make_float2(re, im);
  }
  for (int rI = threadIdx.x; rI < nruns; rI += blockDim.x) {
    uint32_t hi = 0;
    for (int j = L; j < k; j++) hi |= (uint32_t)((rI >> (j - L)) & 1) << d.gpos[j];
    runoff[rI] = hi;
  }
  const CopyCtx cc{runoff, L, nchunk, (uint32_t)lmask};
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int b = 0; b < NBUF; b++) {
      mbar_init(smem_u32(&full[b]), 33);  // 32 copy arrivals + the geometry
      mbar_init(smem_u32(&empty[b]), ncw);
      mbar_init(smem_u32(&freeb[b]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Launched as a programmatic dependent of the previous pass (the
  // specialised kernels): the set-up above overlaps that grid's tail; no
  // thread touches global memory before that grid has completed and its
  // writes are visible. Without the launch attribute this returns at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");

  if (warp == ncw) {
    // --------------------------------------------------------------- loads
    // The load warp takes the CTA's items: its first is blockIdx.x, every
    // later one comes from the launch's counter (taken one item ahead, so
    // the atomic's latency hides behind the tile's copies). CTAs
    // that get through their items faster take more of them, so the CTAs
    // sharing an SM finish together. The warp computes each item's geometry
    // once and publishes it in geo[b]; after the last item it publishes an
    // end marker (node -1) the same way. Lane 0's arrive (release) on
    // full[b] orders geo[b] before the compute and store warps' waits
    // (acquire) on that barrier.
    int64_t it = blockIdx.x;
    uint32_t ahead = 0;  // lane 0: the counter's value for the next item
    for (int i = 0;; i++) {
      const int b = i % NBUF;
      // the item and its geometry do not depend on the buffer: found before
      // waiting for it to be free
      if (i > 0) it = (int64_t)gridDim.x + (int64_t)__shfl_sync(0xffffffffu, ahead, 0);
      const bool last = it >= items;
      if (lane == 0 && !last) ahead = atomicAdd(P.work, 1u);
      ItemGeo g{};
      if (!last) g = Prog::geo(P, it, tiles_log2);
      else g.node = -1;
      if (i >= NBUF && !mbar_wait(smem_u32(&freeb[b]), (uint32_t)((i / NBUF - 1) & 1))) {
        if (lane == 0) {
          abort_flag = 1;
          atomicExch(P.err, 1);
        }
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      if (lane == 0) geo[b] = g;
      if (!last && !d.gen_input) Prog::load_tile(P, g, smem_u32(bufs + b * ntile), lane, cc);
      cp_async_arrive(smem_u32(&full[b]));
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&full[b]));
      if (last) {
        // this CTA takes no more items; the last CTA to get here resets the
        // counters for the next launch (every other CTA has taken its last)
        if (lane == 0) {
          __threadfence();
          if (atomicAdd(P.work + 1, 1u) == gridDim.x - 1u) {
            atomicExch(P.work, 0u);
            atomicExch(P.work + 1, 0u);
          }
        }
        break;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // every tile of this CTA is loaded: the next pass may start its CTAs'
    // set-up where this grid's CTAs have exited
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    return;
  }
  if (warp == ncw + 1) {
    // -------------------------------------------------------------- stores
    for (int i = 0;; i++) {
      const int b = i % NBUF;
      const uint32_t par = (uint32_t)((i / NBUF) & 1);
      // the geometry is readable once full[b] completes (buffer b cannot be
      // refilled before this warp frees it); for a compact output, load the
      // tile's part-map words while the tile is being computed
      bool ok = mbar_wait(smem_u32(&full[b]), par);
      const ItemGeo g = geo[b];
      if (ok && g.node < 0) break;  // end marker
      CompactWord cw{0u, 0u};
      if (ok && P.cmap) cw = compact_word(P, g, lane, 0);
      if (!ok || !mbar_wait(smem_u32(&empty[b]), par) || *(volatile int*)&abort_flag) {
        if (lane == 0) {
          abort_flag = 1;
          atomicExch(P.err, 1);
        }
        break;
      }
      if (P.cmap) compact_store_tile<Prog>(P, g, bufs + b * ntile, lane, cw);
      else Prog::store_tile(P, g, bufs + b * ntile, lane, cc);
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&freeb[b]));
    }
    return;
  }

  // -------------------------------------------------------------- compute
  for (int i = 0;; i++) {
    const int b = i % NBUF;
    float2* sm = bufs + b * ntile;
    const bool timed_out = !mbar_wait(smem_u32(&full[b]), (uint32_t)((i / NBUF) & 1));
    if (compute_bar_or(ncomp, timed_out || *(volatile int*)&abort_flag)) {
      if (threadIdx.x == 0) {
        abort_flag = 1;
        atomicExch(P.err, 1);
      }
      break;
    }
    const ItemGeo g = geo[b];
    if (g.node < 0) break;  // end marker (the same for every compute warp)
    if (d.gen_input) {
      for (int e = threadIdx.x; e < ntile; e += ncomp)
        sm[Prog::swz(e)] = (((uint32_t)e & g.lin_m) == g.lin_v) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
      compute_bar(ncomp);
    } else if (g.lin_m & (uint32_t)lmask) {
      // pins inside a run (the load warp zero-fills the pinned-out runs)
      const uint32_t im = g.lin_m & (uint32_t)lmask, iv = g.lin_v & (uint32_t)lmask;
      for (int e = threadIdx.x; e < ntile; e += ncomp)
        if (((uint32_t)e & im) != iv) sm[Prog::swz(e)] = make_float2(0.f, 0.f);
      compute_bar(ncomp);
    }
    // every compute thread runs the stage program, so that all of them pass
    // the same barrier instructions; threads above 2^(k-R) skip the work
    Prog::run(P, sm, g, w8, ncomp, (int)threadIdx.x < nact);
    if (d.n_stages == 0 && d.post_scale != 1.0f) {
      for (int e = threadIdx.x; e < ntile; e += ncomp) {
        float2 v = sm[e];
        sm[e] = make_float2(v.x * d.post_scale, v.y * d.post_scale);
      }
      compute_bar(ncomp);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&empty[b]));
  }
}


}  // namespace sf
