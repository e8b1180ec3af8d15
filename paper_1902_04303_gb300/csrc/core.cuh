// core.cuh -- shared types of the gwhe library: 64-bit modular arithmetic on
// the GPU, the RNS context, ciphertext handles and launch helpers.
//
// Residues are uint64 limbs of a polynomial in Z_q[X]/(X^N + 1), stored
// limb-major ([poly][limb][N]) and, on the device, in the NTT domain unless a
// buffer is documented as coefficient-domain.  Moduli are below 2^62 so that
// lazy (Harvey) butterflies can keep values in [0, 4q).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

namespace gwhe {

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

constexpr int kMaxMod = 96;     // q-limbs + special primes
constexpr int kMaxRowLimbs = 64;
// rows per item of one batched transform (a ModUp's new limbs of every digit)
constexpr int kMaxRowMap = 192;

// Status codes of the C ABI.
enum Status {
  ST_OK = 0,
  ST_EINVAL = -1,
  ST_ENOMEM = -2,
  ST_ELEVEL = -3,
  ST_ESCALE = -4,
  ST_ENOKEY = -5,
  ST_ETIMEOUT = -6,
  ST_ECUDA = -7,
};

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define GWHE_CUDA(call)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw ::gwhe::Error(::gwhe::ST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define GWHE_CHECK_LAUNCH() GWHE_CUDA(cudaGetLastError())
// every kernel launch of the library goes through this: counts and checks it
#define GWHE_LAUNCHED(ctx, n)         \
  do {                                \
    (ctx)->launches += (n);           \
    GWHE_CUDA(cudaGetLastError());    \
  } while (0)

#define GWHE_REQUIRE(cond, code, msg)                    \
  do {                                                   \
    if (!(cond)) throw ::gwhe::Error((code), (msg));     \
  } while (0)

#if defined(__CUDACC__)
// Launch of a kernel that begins with pdl_wait() (below) on stream st, with
// programmatic stream serialisation: its CTAs may be scheduled while the
// previous kernel on the stream drains, which hides the launch gap between
// dependent kernels.  Every argument of the kernel must be given.
template <typename... KArgs, typename... Args>
inline void pdl_launch(cudaStream_t st, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       Args&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  GWHE_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}
#endif

// Per-modulus constants.  R = 2^64 mod q with its Shoup companion, and the
// 64-bit Barrett factor floor(2^64 / q).
struct DevMod {
  u64 q, twoq, R, Rsh, mu;
};

// ---------------------------------------------------------------- device math
#if defined(__CUDACC__)
__device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }

// Shoup product x*w mod q for a constant w < q with wsh = floor(w 2^64 / q);
// valid for any x < 2^64, result in [0, 2q).
__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 wsh, u64 q) {
  u64 h = __umul64hi(x, wsh);
  return x * w - h * q;
}
__device__ __forceinline__ u64 shoup(u64 x, u64 w, u64 wsh, u64 q) {
  return csub(shoup_lazy(x, w, wsh, q), q);
}

// Shoup product with an estimated quotient, for the NTT butterflies.  With
// y = y1 2^32 + y0 and w' = s1 2^32 + s0 (w' = floor(w 2^64 / q)), the
// quotient floor(y w' / 2^64) is estimated by e = y1 s1 + hi32(y1 s0) +
// hi32(y0 s1): the dropped terms (the low words of the cross products and
// y0 s0) sum to less than 3 * 2^64, so e is at most 2 below the exact quotient
// and never above it.  The Shoup remainder y w - quotient q lies in [0, 2q)
// for any y < 2^64, hence r = y w - e q lies in [0, 4q).  The low word is
// formed as y w + e (2^64 - q) mod 2^64 with nq = 2^64 - q, from 32-bit
// multiply-adds.
__device__ __forceinline__ u64 shoup_est(u64 y, u64 w, u64 wsh, u64 nq) {
  u64 r;
  asm("{\n\t"
      ".reg .u32 y0, y1, w0, w1, s0, s1, h1, h2, cy, e0, e1, n0, n1, r0, r1;\n\t"
      ".reg .u64 e, t;\n\t"
      "mov.b64 {y0, y1}, %1;\n\t"
      "mov.b64 {w0, w1}, %2;\n\t"
      "mov.b64 {s0, s1}, %3;\n\t"
      "mov.b64 {n0, n1}, %4;\n\t"
      "mul.hi.u32 h1, y1, s0;\n\t"
      "mul.hi.u32 h2, y0, s1;\n\t"
      "add.cc.u32 h1, h1, h2;\n\t"
      "addc.u32 cy, 0, 0;\n\t"
      "mov.b64 t, {h1, cy};\n\t"
      "mad.wide.u32 e, y1, s1, t;\n\t"
      "mov.b64 {e0, e1}, e;\n\t"
      "mul.wide.u32 t, y0, w0;\n\t"
      "mad.wide.u32 t, e0, n0, t;\n\t"
      "mov.b64 {r0, r1}, t;\n\t"
      "mad.lo.u32 r1, y0, w1, r1;\n\t"
      "mad.lo.u32 r1, y1, w0, r1;\n\t"
      "mad.lo.u32 r1, e0, n1, r1;\n\t"
      "mad.lo.u32 r1, e1, n0, r1;\n\t"
      "mov.b64 %0, {r0, r1};\n\t"
      "}"
      : "=l"(r)
      : "l"(y), "l"(w), "l"(wsh), "l"(nq));
  return r;
}

// Programmatic dependent launch: a kernel started by pdl_launch may become
// resident while the kernel before it on the stream is still finishing.  It
// calls pdl_wait() before its first memory access (the wait returns once the
// previous kernel has completed and its writes are visible; without a
// programmatic predecessor it returns at once) and then pdl_trigger(), which
// lets the next kernel on the stream start its own launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Harvey-style lazy butterflies on [0, 8q) (q < 2^60, so 8q < 2^63), with the
// estimated Shoup product t in [0, 4q) and q4 = 4q:
//   Cooley-Tukey:     a = x mod' 4q in [0, 4q); x = a + t, y = a - t + 4q
//   Gentleman-Sande:  x = (x + y) mod' 4q; y = Shoup(x - y + 4q) in [0, 4q)
// (mod' = one conditional subtraction).  Both keep every value below 8q.
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, u64 w, u64 wsh, u64 q4, u64 nq) {
  const u64 a = csub(x, q4);
  const u64 t = shoup_est(y, w, wsh, nq);
  x = a + t;
  y = a - t + q4;
}
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, u64 w, u64 wsh, u64 q4, u64 nq) {
  const u64 s = x + y;
  const u64 d = x - y + q4;
  x = csub(s, q4);
  y = shoup_est(d, w, wsh, nq);
}
// [0, 8q) -> [0, q)
__device__ __forceinline__ u64 reduce_8q(u64 x, u64 q) {
  return csub(csub(csub(x, 4 * q), 2 * q), q);
}
// y w mod q in [0, q) for any y < 2^64: the estimated Shoup product (in
// [0, 4q), fewer 32-bit multiplies than the exact quotient) and two
// conditional subtractions
__device__ __forceinline__ u64 shoup_est_canon(u64 y, u64 w, u64 wsh, u64 q, u64 nq) {
  return csub(csub(shoup_est(y, w, wsh, nq), 2 * q), q);
}

// (hi 2^64 + lo) mod q: hi 2^64 = hi R (mod q) by a Shoup product, lo by a
// 64-bit Barrett step (quotient estimate off by at most one).
__device__ __forceinline__ u64 reduce128(u64 lo, u64 hi, const DevMod& m) {
  u64 a = csub(shoup_lazy(hi, m.R, m.Rsh, m.q), m.q);
  u64 b = csub(lo - __umul64hi(lo, m.mu) * m.q, m.q);
  return csub(a + b, m.q);
}
__device__ __forceinline__ u64 mulmod(u64 a, u64 b, const DevMod& m) {
  return reduce128(a * b, __umul64hi(a, b), m);
}
__device__ __forceinline__ u64 reduce64(u64 x, const DevMod& m) {
  return csub(x - __umul64hi(x, m.mu) * m.q, m.q);
}
__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 q) {
  u64 s = a + b;
  return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulator: safe for up to 128 products of residues below 2^60.
struct Acc128 {
  u64 lo, hi;
};
// a += v on 128 bits
__device__ __forceinline__ void add128(Acc128& a, u64 v) {
  a.lo += v;
  a.hi += a.lo < v;
}
// a += x * y on 128 bits, as a schoolbook product of 32-bit halves with
// multiply-add carry chains: the x0 y0 and x1 y1 partial products go to words
// 0-1 and 2-3, the two cross products to words 1-2.
__device__ __forceinline__ void mac128(Acc128& a, u64 x, u64 y) {
  const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
  const uint32_t y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
  uint32_t r0 = (uint32_t)a.lo, r1 = (uint32_t)(a.lo >> 32);
  uint32_t r2 = (uint32_t)a.hi, r3 = (uint32_t)(a.hi >> 32);
  asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
      "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
      "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
      "madc.hi.u32 %3, %5, %7, %3;\n\t"
      "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
      "addc.u32 %3, %3, 0;\n\t"
      "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
      "addc.u32 %3, %3, 0;"
      : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3)
      : "r"(x0), "r"(x1), "r"(y0), "r"(y1));
  a.lo = ((u64)r1 << 32) | r0;
  a.hi = ((u64)r3 << 32) | r2;
}

#endif  // __CUDACC__

// Maps the rows of a batched transform to memory and moduli:
// row r -> poly r / nl, limb r % nl at data + (poly * poly_stride + off[limb]) * N,
// modulus index pidx[limb].
struct RowMap {
  int npoly;
  int nl;
  int poly_stride;
  uint16_t off[kMaxRowMap];
  uint8_t pidx[kMaxRowMap];
};

// Tables of the negacyclic NTT for one modulus index u, each of length N:
// psi[i] = (psi^brv(i), Shoup companion), ipsi[i] = (psi^-brv(i), companion),
// interleaved so that one 16-byte load fetches a twiddle and its companion.
// psiB / ipsiB (N = 2^16 only): the twiddles of the row pass's stages 12-15
// (local stages 4-7 of the 8 + 8 split with 16 residues per thread),
// transposed so that a warp's loads are contiguous: for local stage sp,
// row g, the thread r of the row and its j-th distinct twiddle j < 2^(sp-4),
// entry kTwB[sp] + g 2^sp + 16 j + r = psi[2^(8+sp) + g 2^sp + r 2^(sp-4) + j].
constexpr int kTwBPerMod = 256 * (16 + 32 + 64 + 128);
struct NttTables {
  const ulonglong2* psi;
  const ulonglong2* ipsi;
  const ulonglong2* psiB;   // [nmod][kTwBPerMod] or null
  const ulonglong2* ipsiB;
  const u64* ninv;     // [nmod] N^-1 mod q_u
  const u64* ninv_sh;  // [nmod]
  const DevMod* mod;   // [nmod]
  // [nmod] ipsi[1] N^-1 mod q_u and its Shoup companion: the last inverse
  // stage's twiddle with the factor N^-1 merged in
  const ulonglong2* iw1n;
};

struct Context;

// A ciphertext (npoly = 2) or a tensor (npoly = 3) in the NTT domain on the
// device: poly p, limb i at d + (p * cap + i) * N.
struct Ct {
  Context* ctx = nullptr;
  u64* d = nullptr;
  int npoly = 2;
  int cap = 0;
  int l = 0;
  double scale = 1.0;
  bool owned = true;
  ~Ct();
  u64* poly(int p) const;
  u64* limb(int p, int i) const;
};
typedef std::unique_ptr<Ct> CtPtr;

// One family of a switching key, for the key switches that use k special
// primes (the levels l with K_l = k, up to lmax): NTT domain,
// [dk][2][lmax + k][N] with dk = ceil(lmax / alpha) digits; rows are
// q_0..q_{lmax-1} then p_0..p_{k-1}.
constexpr int kMaxSpecial = 16;
struct Ksk {
  u64* d = nullptr;
  int k = 0, lmax = 0, dk = 0;
  int rows() const { return lmax + k; }
};
// A switching key: its families, indexed by the special-prime count k.
struct KeySet {
  Ksk fam[kMaxSpecial + 1];
};

struct Params {
  int logN, L, q0_bits, scale_bits, K, sp_bits, dnum;
};

struct ConvTable {  // fast base conversion constants, on the device
  const u64* dev;   // [n_in] hinv, [n_in] hinv_sh, [n_in][n_out] hmod
  // [n_in][2]: (hinv N^-1, Shoup) and (ipsi[1] hinv N^-1, Shoup) mod the
  // input's modulus, for an inverse transform whose output is the
  // conversion's input already multiplied by hinv (ntt_inverse's iscale)
  const ulonglong2* iscale = nullptr;
  int n_in, n_out;
  int in_lo;                          // first input q-limb (ModUp digits)
  std::vector<uint8_t> in_pidx;       // modulus index of each input limb (empty: in_lo + i)
  std::vector<uint8_t> out_pidx;      // modulus index of each output limb
  std::vector<uint16_t> out_limb;     // position of each output limb in the extended basis
};

// Kernel classes timed by the optional profiler (CUDA events on the stream).
enum ProfCat {
  PROF_NTT = 0,
  PROF_KS_INNER = 1,
  PROF_TENSOR_MAC = 2,
  PROF_BASECONV = 3,
  PROF_ELEMWISE = 4,
  PROF_ENCODE = 5,
  PROF_SAMPLE = 6,
  PROF_NCAT = 7
};
struct ProfRec {
  cudaEvent_t a, b;
  double bytes;
  int cat;
};
struct Prof {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
};

struct Context {
  // a child context (ctx_child) shares its parent's tables and keys
  // read-only and owns only its stream, caches and counters
  const Context* parent = nullptr;
  // pinned host staging buffers of the genotype columns (grow-only, kept
  // across calls: pinned allocation and release are slow and synchronising)
  void* pin_stage[2] = {nullptr, nullptr};
  size_t pin_stage_bytes = 0;
  // pinned block for one job's Dup(M_j) in the host tier (grow-only; lent
  // to one job at a time, others allocate their own)
  void* pin_state = nullptr;
  size_t pin_state_bytes = 0;
  bool pin_state_lent = false;
  Params P;
  // the CUDA device the context's tables, keys and pool live on (current at
  // creation); every call must be made with this device current
  int device = 0;
  // device address of the allocation-free key switch's static scratch array
  // on that device (resolved at creation, see noalloc.cu)
  u64* noalloc_scratch = nullptr;
  int N = 0, logN = 0, alpha = 0, nmod = 0;
  int ntt_variant = 4;         // shape of the N = 2^16 transform (kNttVariants;
                               // 4 = the fastest measured on GB300, see gwhe_autotune)
  int ntt_variant_small = 4;   // the shape for launches below kNttSmallRows rows
  u64 seed = 0;
  cudaStream_t stream = 0;
  std::vector<u64> mod;        // [L + K]: q_0..q_{L-1}, p_0..p_{K-1}
  std::vector<DevMod> hmod;
  DevMod* d_mod = nullptr;
  ulonglong2 *d_psi = nullptr, *d_ipsi = nullptr;
  ulonglong2 *d_psiB = nullptr, *d_ipsiB = nullptr;  // row-pass twiddles, N = 2^16
  u64 *d_ninv = nullptr, *d_ninv_sh = nullptr;
  ulonglong2* d_iw1n = nullptr;
  // rescale: q_{l-1}^-1 mod q_i for every level l and i < l - 1 (value, Shoup)
  u64* d_rescale = nullptr;    // [L][L][2]
  // key switches at level l use the first ks_k[l] special primes (fewest
  // whose product exceeds the level's widest digit by 24 bits, else all K);
  // key_lmax[k] = the highest level using k (0 if none)
  int ks_k[kMaxRowLimbs + 1] = {};
  int key_lmax[kMaxSpecial + 1] = {};
  // ModUp tables per (level l, digit j); ModDown tables and P_k^-1 per k
  std::map<std::pair<int, int>, ConvTable> modup;
  ConvTable moddown[kMaxSpecial + 1];
  u64* d_pinv[kMaxSpecial + 1] = {};  // [L][2] P_k^-1 mod q_i (value, Shoup)
  // relinearisation fused with rescale at level l: conversion from
  // {p_0..p_{K_l-1}, q_{l-1}} to q_0..q_{l-2} and the constants of the
  // division by P' = P q_{l-1} (see k_fused_prep / k_fused_combine)
  ConvTable fused[kMaxRowLimbs + 1];
  u64* d_fused[kMaxRowLimbs + 1] = {};
  u64* d_conv_store = nullptr; // backing store of all conversion tables
  ulonglong2* d_iscale_store = nullptr;  // backing store of the iscale arrays
  // ModUp at level l: the iscale pairs of all l limbs (each from its digit's
  // table), in limb order, for the one inverse transform of every digit
  const ulonglong2* modup_iscale[kMaxRowLimbs + 1] = {};
  // encoding procedure tables
  double2* d_fftW_dec = nullptr;
  longlong2* d_fftWq = nullptr;   // [M/2] encoding twiddles, 62 fractional bits
  longlong2* d_fftTq = nullptr;   // [M]
  double2* d_fftT_dec = nullptr;
  int* d_slot_u = nullptr;        // [M] u_j
  int* d_slot_inv = nullptr;      // [M] slot j with bitrev(u_j) = p, for each p
  // keys
  u64* d_sk = nullptr;            // [L+K][N] NTT domain
  u64* d_pk = nullptr;            // [2][L][N] NTT domain (b, a)
  std::map<u32, KeySet> ksk;      // key id -> switching key
  bool have_keys = false;
  // encoded public plaintexts (masks), keyed by (kind, index, level, scale):
  // the plaintext, the stream that encoded it and an event recorded after
  // the encoding (a use on another stream of the context waits for it)
  struct Mask {
    u64* pt;
    cudaStream_t stream;
    cudaEvent_t done;
  };
  std::map<std::tuple<int, long, int, double>, Mask> masks;
  long ks_count = 0;              // key switches issued (relinearisations + automorphisms)
  long launches = 0;              // kernels launched
  long ks_by_level[kMaxRowLimbs + 1] = {};  // key switches per level
  Prof prof;
  std::string last_error;
  NttTables tables() const {
    return NttTables{d_psi, d_ipsi, d_psiB, d_ipsiB, d_ninv, d_ninv_sh, d_mod, d_iw1n};
  }
};

// shapes of the N = 2^16 transform compiled in (identical results)
constexpr int kNttVariants = 7;
// launches with fewer rows (a few waves of CTAs or less) use their own shape
constexpr int kNttSmallRows = 128;

// the family of key id that a switch at level l uses (ST_ENOKEY if absent)
const Ksk& key_family(const Context* c, u32 key_id, int l);

// ---------------------------------------------------------------- host helpers
// params.cpp
int gen_primes(int logN, int L, int q0_bits, int scale_bits, int K, int sp_bits, u64* q, u64* p);
u64 host_mulmod(u64 a, u64 b, u64 m);
u64 host_powmod(u64 a, u64 e, u64 m);
u64 host_inv(u64 a, u64 m);
u64 find_psi(u64 q, int logN);
u64 shoup_companion(u64 w, u64 q);
DevMod make_devmod(u64 q);
void fft_twiddles(int logN, int sign, double* W, double* T);
int bitrev_host(int x, int bits);

// Records CUDA events around the launches in its scope when profiling is on;
// bytes = the algorithmic traffic of those launches.
struct ProfScope {
  Context* c;
  int cat;
  double bytes;
  cudaEvent_t a = nullptr;
  ProfScope(Context* c_, int cat_, double bytes_);
  ~ProfScope();
};
void prof_read(Context* c, double* ms, double* bytes, long* count);

// noalloc.cu: the static scratch array's address on the current device
// (loads the array's module and commits its memory there)
u64* noalloc_scratch_lookup();

// ST_OK when current_device is the context's device, else ST_EINVAL
int device_check(int context_device, int current_device);
// the context's device must be current (ST_EINVAL otherwise)
void require_device(const Context* c);

// device memory helpers (stream-ordered pool)
u64* dalloc_u64(Context* c, size_t words);
void dfree(Context* c, void* p);
void* dalloc_bytes(Context* c, size_t bytes);

// ntt.cu
void ntt_forward(Context* c, u64* data, const RowMap& rm);
// ModDown's last step fused into a forward transform: data holds the
// converted limbs conv [cnt][2][l][N] (coefficient domain); instead of
// writing NTT(conv) back, the row pass writes
//   out_p[item][i] = (acc[item][p][i] - NTT(conv)[item][p][i]) P^-1 (+ add_p[item][i])
// with acc [cnt][2][l + K][N] (extended basis, NTT domain), pinv = the
// (P^-1 mod q_i, Shoup companion) pairs, add0/add1 optional.  data is left
// partly transformed.  Rings below 2^12 return false (not fused).
struct MdEpi {
  const u64* acc;
  int l, K;
  u64 *out0, *out1;
  size_t o_stride;
  const u64 *add0, *add1;
  size_t a0_stride, a1_stride;
  const u64* pinv;
};
bool ntt_forward_moddown(Context* c, u64* data, int cnt, const MdEpi& epi);
// iscale (device, optional): [rm.nl][2] pairs (s N^-1, Shoup), (ipsi[1] s
// N^-1, Shoup) per row-map limb; the output is the inverse transform times s
// (canonical residues), the factor merged into the last stage
void ntt_inverse(Context* c, u64* data, const RowMap& rm, const ulonglong2* iscale = nullptr);
RowMap rows_q(int npoly, int l, int poly_stride);  // limbs 0..l-1 of q-primes

}  // namespace gwhe
