// Device-side records of a fused pass launch, shared by the library (nvcc,
// host and device) and by the run-time specialised pass kernels (NVRTC), so
// both see one layout. Plain types only; nothing here may need a host header
// under NVRTC.
#pragma once

#if defined(__CUDACC_RTC__)
namespace sf {
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
}  // namespace sf
#else
#include <cstdint>
#endif

#if defined(__CUDACC__)
#define SF_HD __host__ __device__
#else
#define SF_HD
#endif

namespace sf {

// ------------------------------------------------------------ device limits
constexpr int MAX_K = 14;          // tile bits (2^14 complex64 = 128 KiB)
constexpr int MAX_R = 5;           // register bits per thread
constexpr int MAX_PINS = 12;
constexpr int MAX_STAGES = 48;
constexpr int MAX_OPS = 160;
constexpr int MAX_PHASE_GROUPS = 40;
constexpr int MAX_CZ_PER_GROUP = 40;
constexpr int MAX_SEL_PER_GROUP = 8;
constexpr int MAX_SHIFTS = 16;
constexpr int MAX_MATS = 640;      // float2 entries of matrices per pass
constexpr int MAX_NODES = 128;     // nodes per pass launch
constexpr int MAX_CROSS = 64;
constexpr int MAX_DEFER = 4;
constexpr int GATHER_FINALS = 64;  // finals per gather launch

// Device op codes (applied to a thread's register block; bits are
// register-local indices a, b in [0, r)).
enum DevOpCode : int32_t {
  DOP_H = 1,      // [[1,1],[1,-1]] (scale 1/sqrt2 deferred)
  DOP_XH = 2,     // [[1,-i],[-i,1]] = sqrt2 e^{-i pi/4} X^1/2 (factor deferred)
  DOP_YH = 3,     // [[1,-1],[1,1]] = sqrt2 e^{-i pi/4} Y^1/2 (factor deferred)
  DOP_G1 = 4,     // general 2x2, mats[arg..arg+4)
  DOP_G1SEL = 5,  // 2x2 chosen by the digit of cross gate xi: mats[arg + 4*d ..]
  DOP_G2 = 6,     // general 4x4 on (a = high bit of the basis index, b = low)
  DOP_PHASE = 7,  // phase group phases[arg] (mod-8 powers of e^{i pi/4})
  DOP_DMUL = 8,   // diagonal (f0, f1) on global half position a: mats[arg], mats[arg+1]
  DOP_DMULSEL = 9 // as DMUL, pair chosen by digit of cross gate xi: mats[arg + 2*d ..]
};

struct DevOp {
  int32_t code;
  int32_t a, b;
  int32_t xi;
  int32_t arg;
};

// A group of diagonal gates whose product is exp(i pi/4 * k(idx)), idx the
// global index inside the half state, prepared for one register stage: with
// idx = gfix | (register bits), k is a quadratic form in the register bits
//   k = k0(gfix) + sum_j w_j i_j + 4 sum_{j<l, partners} i_j i_l   (mod 8)
//   k0 = popc(gfix&m1) + 2 popc(gfix&m2) + 4 popc(gfix&m4)
//        + 4 sum_s popc(gfix & (gfix >> sh_s) & shm_s) + [selected weights]
//   w_j = wstat_j + 4 popc(gfix & czf_j) + [selected weights]
struct DevPhaseGroup {
  uint32_t m1, m2, m4;       // weights (bits 1,2,4) of the fixed positions
  uint8_t wstat[MAX_R];      // weight of register bit j from one-qubit phases
  uint8_t czq[MAX_R];        // CZ partners of register bit j among register bits
  uint32_t czf[MAX_R];       // CZ partners of register bit j among fixed positions
  int32_t nsh;               // CZ pairs between fixed positions, by shift
  uint8_t sh[MAX_SHIFTS];
  uint32_t shm[MAX_SHIFTS];
  int32_t nsel;              // path-selected phases (the B-side Z^b of Eq. 1)
  struct {
    int8_t pos, xi, reg;     // reg: register bit index or -1
    uint8_t w[4];            // weight per digit value
  } sel[MAX_SEL_PER_GROUP];
};

struct DevPin {
  int8_t pos;  // global half position
  int8_t xi;   // -1: constant v[0]; else value v[digit of cross gate xi]
  uint8_t v[4];
};

struct DevStage {
  int32_t r;
  int8_t rbit[MAX_R];  // tile-local bit index of register bit j
  int8_t tpos[9];      // tile-local bit of thread-index bit i (k - r <= 9 of them)
  int8_t tg[9];        // global position of thread-index bit i
  int32_t op_begin, op_end;
};

struct DevPass {
  int32_t m, k, L;
  int32_t R;                 // register bits of every stage (threads = 2^(k-R))
  int32_t n_free;            // inactive bits free to enumerate tiles
  int8_t freepos[32];        // their global positions, ascending
  int8_t gpos[MAX_K];        // tile-local bit j -> global position
  int32_t n_pin_in;
  DevPin pin_in[MAX_PINS];   // all pins of the input (zero outside)
  int32_t n_pin_out;
  DevPin pin_out[MAX_PINS];  // pins of the output (positions not written)
  int32_t gen_input;         // input = root state: 1 on live entries
  float post_scale;          // exact power of two applied at store
  int32_t n_stages;
};

struct PassNode {
  const void* in;  // float2*, ignored when gen_input
  void* out;
  uint64_t path;   // path id bits that select digits
};

struct PassLaunch {
  DevPass pass;
  DevStage stages[MAX_STAGES];
  DevOp ops[MAX_OPS];
  DevPhaseGroup phases[MAX_PHASE_GROUPS];
  float mats[2 * MAX_MATS];
  uint8_t xshift[MAX_CROSS];
  uint8_t xbits[MAX_CROSS];
  int* err;        // set to 1 if a bounded wait gave up
  // Work distribution: work[0] hands out the items after each CTA's first
  // (item = gridDim.x + atomicAdd(work, 1)), work[1] counts the CTAs that
  // have taken their last; the last of them sets both back to zero, so they
  // are zero at the start of every launch (the caller zeroes them once).
  uint32_t* work;
  // Compact output (final passes whose result only the gather reads): null =
  // every live amplitude is written at its index. Otherwise only requested
  // parts are written. A part is a tile's share of one block of the gather
  // (2^ctl consecutive tile elements: positions 0..ctl-1); parts are numbered
  // tile-major, P = tile * 2^(k-ctl) + u for part u of the tile, and part P
  // goes to out + slot(P) * 2^ctl, slot(P) = requested parts below P. cmap
  // holds per 32 parts the pair (bitmap word, requested parts in earlier
  // words), so a tile's parts are consecutive bits of the map.
  const uint32_t* cmap;
  int32_t ctl;
  int32_t cpad;
  int32_t n_nodes;
  PassNode nodes[MAX_NODES];
};


// The bits of x at the set positions of mask, packed from bit 0 up in
// ascending position order.
SF_HD inline uint32_t pext32(uint32_t x, uint32_t mask) {
  uint32_t r = 0, b = 1;
  while (mask) {
    const uint32_t low = mask & (0u - mask);
    if (x & low) r |= b;
    b <<= 1;
    mask ^= low;
  }
  return r;
}

// Shared-memory layout of a tile: element e lives at swz(e), a linear XOR
// swizzle that folds index bits 4..12 into bits 1..3. It keeps 16-byte
// chunks (element pairs) intact for the copy warps and, being linear,
// swz(a ^ b) = swz(a) ^ swz(b), so register stages address amplitude i of a
// thread as swz(thread part) ^ swz(register part); it spreads the stages'
// strided accesses over the shared-memory banks.
SF_HD inline uint32_t swz(uint32_t e) {
  const uint32_t x = e >> 4;
  return e ^ (((x ^ (x >> 3) ^ (x >> 6)) & 7u) << 1);
}

}  // namespace sf
