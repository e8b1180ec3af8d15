// ntt.cu -- batched negacyclic NTT / inverse NTT over RNS limbs.
//
// Forward transform (merged psi twist, Cooley-Tukey): for stage s = 0..logN-1
// with m = 2^s blocks of half-size t = N / 2m, block i pairs (a[j], a[j+t]) with
// twiddle psi^brv(m+i); the output slot j holds a(psi^(2 brv(j) + 1)).  The
// inverse runs the Gentleman-Sande butterflies in reverse stage order with the
// inverse twiddles and multiplies by N^-1.  Both keep lazy ranges below 8q
// between stages (and between the two passes) and return canonical residues
// in [0, q).
//
// Layout for N = 2^12..2^17: the row is viewed as a 2^LA x 2^LB matrix
// (element h * 2^LB + c).  Pass A runs the first LA stages as independent
// 2^LA-point transforms down the columns, pass B the last LB stages along the
// rows.  In each pass a 256-thread CTA owns 4096 residues: 16 per thread, the
// first four local stages in registers in a strided layout (coalesced global
// loads), a shared-memory transpose to a contiguous layout for the remaining
// stages, and a transpose back for coalesced stores; the 9-stage pass of
// N = 2^17 uses 128-thread CTAs with 32 residues per thread (5 + 4 stages).
// Each residue is read and written once per pass.  Smaller rings use one CTA
// per row in shared memory.
#include <cooperative_groups.h>

#include <mutex>

#include "core.cuh"

namespace gwhe {

// One pass of the two-pass transform.  LS = log2 of this pass's sub-transform
// size; the other dimension has 2^(LOGN-LS) entries.  PASSA: sub-transforms
// are columns (stride 2^(LOGN-LS)), global stages 0..LS-1; otherwise rows
// (contiguous), global stages LOGN-LS..LOGN-1.  A CTA of NT threads holds E
// residues per thread (LS <= 2 log2 E): log2 E stages in registers in a
// strided layout, a shared-memory transpose to a contiguous layout for the
// remaining stages, and a transpose back for coalesced stores.
// MD (forward row pass only): ModDown epilogue, see ntt_forward_moddown.
template <int LOGN, int LS, bool PASSA, bool FWD, int E = 16, int NT = 256, int MB = 4,
          bool MD = false>
__global__ void __launch_bounds__(NT, MB) k_ntt_pass(u64* __restrict__ data, const RowMap rm,
                                                  const NttTables tb, const int groups_per_row,
                                                  const MdEpi epi,
                                                  const ulonglong2* __restrict__ iscale) {
  pdl_wait();
  pdl_trigger();
  static_assert(!MD || (FWD && !PASSA), "the ModDown epilogue ends a forward transform");
  constexpr int S = 1 << LS;
  constexpr int LE = E == 16 ? 4 : 5;  // log2 E
  static_assert(E == 16 || E == 32, "16 or 32 residues per thread");
  static_assert(LS <= 2 * LE && LS > LE, "sub-transform size out of range");
  constexpr int TPS = S / E;          // threads per sub-transform
  constexpr int G = NT / TPS;         // sub-transforms per CTA
  constexpr int LC = LOGN - LS;       // log2 of the other dimension
  // padding keeps the strided and contiguous accesses free of bank conflicts:
  // one word per E residues, and a row pitch that spreads the sub-transforms
  // of a half-warp over distinct 64-bit banks (G < 16 column sub-transforms
  // per CTA need a pitch of 2 mod 16, G = 16 one of 1 mod 16)
  constexpr bool PADE = !PASSA || E == 32 || G < 16;
  constexpr int PADS = PADE ? (S + S / E + (E == 32 ? 1 : (PASSA ? 2 : 0))) : (S + 1);
  constexpr int S0 = PASSA ? 0 : LC;  // global index of local stage 0
  __shared__ u64 sm[G * PADS];

  const int row = blockIdx.x / groups_per_row;
  const int grp = blockIdx.x - row * groups_per_row;
  const int poly = row / rm.nl;
  const int limb = row - poly * rm.nl;
  const int u = rm.pidx[limb];
  u64* base = data + ((size_t)poly * rm.poly_stride + rm.off[limb]) * ((size_t)1 << LOGN);
  const u64 q = tb.mod[u].q, q4 = 4 * q, nq = 0 - q;
  const ulonglong2* W = (FWD ? tb.psi : tb.ipsi) + ((size_t)u << LOGN);

  const int t = threadIdx.x;
  const int lg = PASSA ? (t % G) : (t / TPS);
  const int r = PASSA ? (t / G) : (t % TPS);
  const int g = grp * G + lg;

  auto gaddr = [&](int e) -> size_t {
    return PASSA ? (((size_t)e << LC) + g) : (((size_t)g << LS) + e);
  };
  auto sidx = [&](int e) -> int { return PADE ? (lg * PADS + e + (e >> LE)) : (lg * PADS + e); };
  auto tw = [&](int s_local, int e) -> int {  // twiddle index for the pair led by e
    const int s = S0 + s_local;
    return (1 << s) + (PASSA ? 0 : (g << s_local)) + (e >> (LS - s_local));
  };
  // the row pass of the 8 + 8 split at 16 residues per thread reads its
  // contiguous-layout stages from the transposed table (coalesced per warp)
  constexpr bool TWB = !PASSA && LOGN == 16 && LS == 8 && E == 16;
  const ulonglong2* WB = TWB ? (FWD ? tb.psiB : tb.ipsiB) + (size_t)u * kTwBPerMod : nullptr;
  auto twb = [&](int sp, int m) -> ulonglong2 {  // stage sp >= 4, pair led by E r + m
    const int off = 256 * ((1 << sp) - 16);     // sum over the earlier stages 4..sp-1
    return __ldg(WB + off + (g << sp) + ((m >> (8 - sp)) << 4) + r);
  };

  u64 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = base[gaddr(r + TPS * m)];

  if (FWD) {
#pragma unroll
    for (int sp = 0; sp < LE; ++sp) {
      const int st = (E / 2) >> sp;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const int idx = tw(sp, TPS * m);
        const ulonglong2 w = __ldg(W + idx);
        ct_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sidx(r + TPS * m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sidx(E * r + m)];
#pragma unroll
    for (int sp = LE; sp < LS; ++sp) {
      const int st = S >> (sp + 1);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = TWB ? twb(sp, m) : __ldg(W + tw(sp, E * r + m));
        ct_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sidx(E * r + m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sidx(r + TPS * m)];
    if (!PASSA) {
#pragma unroll
      for (int m = 0; m < E; ++m) x[m] = reduce_8q(x[m], q);
    }
    if (MD) {
      // row = (item, poly p, limb) of conv [cnt][2][l][N]
      const size_t N = (size_t)1 << LOGN;
      const int item = poly >> 1, p = poly & 1;
      const u64* a = epi.acc + ((size_t)item * 2 * (epi.l + epi.K) + (size_t)p * (epi.l + epi.K) +
                                limb) * N;
      u64* o = (p ? epi.out1 : epi.out0) + item * epi.o_stride + (size_t)limb * N;
      const u64* ad = p ? epi.add1 : epi.add0;
      if (ad) ad += item * (p ? epi.a1_stride : epi.a0_stride) + (size_t)limb * N;
      const u64 pi = epi.pinv[2 * limb], pish = epi.pinv[2 * limb + 1];
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const size_t k = gaddr(r + TPS * m);
        u64 v = shoup_est_canon(submod(a[k], x[m], q), pi, pish, q, nq);
        if (ad) v = addmod(v, ad[k], q);
        o[k] = v;
      }
      return;
    }
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sidx(r + TPS * m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sidx(E * r + m)];
#pragma unroll
    for (int sp = LS - 1; sp >= LE; --sp) {
      const int st = S >> (sp + 1);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = TWB ? twb(sp, m) : __ldg(W + tw(sp, E * r + m));
        gs_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sidx(E * r + m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sidx(r + TPS * m)];
#pragma unroll
    for (int sp = LE - 1; sp >= (PASSA ? 1 : 0); --sp) {
      const int st = (E / 2) >> sp;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const int idx = tw(sp, TPS * m);
        const ulonglong2 w = __ldg(W + idx);
        gs_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    if (PASSA) {
      // global stage 0 (every pair on twiddle index 1) with the factor N^-1
      // (times the row's scale s, if given) merged in: x = (x + y) s N^-1,
      // y = (x - y) (w s N^-1), both Shoup products of inputs below 8q made
      // canonical in [0, q)
      u64 ni, nish;
      ulonglong2 wn;
      if (iscale) {
        const ulonglong2 a = iscale[2 * limb];
        ni = a.x;
        nish = a.y;
        wn = iscale[2 * limb + 1];
      } else {
        ni = tb.ninv[u];
        nish = tb.ninv_sh[u];
        wn = tb.iw1n[u];
      }
      constexpr int st = E / 2;
#pragma unroll
      for (int m = 0; m < st; ++m) {
        const u64 a = x[m], b = x[m + st];
        x[m] = shoup_est_canon(a + b, ni, nish, q, nq);
        x[m + st] = shoup_est_canon(a - b + q4, wn.x, wn.y, q, nq);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < E; ++m) base[gaddr(r + TPS * m)] = x[m];
}

// Whole row in shared memory (N <= 2^11), one CTA per row.
template <bool FWD>
__global__ void __launch_bounds__(256) k_ntt_small(u64* __restrict__ data, const RowMap rm,
                                                   const NttTables tb, const int logN,
                                                   const ulonglong2* __restrict__ iscale) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ u64 sh[];
  const int N = 1 << logN;
  const int row = blockIdx.x;
  const int poly = row / rm.nl;
  const int limb = row - poly * rm.nl;
  const int u = rm.pidx[limb];
  u64* base = data + ((size_t)poly * rm.poly_stride + rm.off[limb]) * (size_t)N;
  const u64 q = tb.mod[u].q, q4 = 4 * q, nq = 0 - q;
  const ulonglong2* W = (FWD ? tb.psi : tb.ipsi) + ((size_t)u << logN);
  for (int i = threadIdx.x; i < N; i += blockDim.x) sh[i] = base[i];
  __syncthreads();
  const int half = N >> 1;
  if (FWD) {
    for (int s = 0; s < logN; ++s) {
      const int lt = logN - 1 - s;  // log2 of t
      for (int b = threadIdx.x; b < half; b += blockDim.x) {
        const int i = b >> lt;
        const int j = (i << (lt + 1)) + (b & ((1 << lt) - 1));
        const int idx = (1 << s) + i;
        const ulonglong2 w = W[idx];
        ct_bfly(sh[j], sh[j + (1 << lt)], w.x, w.y, q4, nq);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) base[i] = reduce_8q(sh[i], q);
  } else {
    for (int s = logN - 1; s >= 0; --s) {
      const int lt = logN - 1 - s;
      for (int b = threadIdx.x; b < half; b += blockDim.x) {
        const int i = b >> lt;
        const int j = (i << (lt + 1)) + (b & ((1 << lt) - 1));
        const int idx = (1 << s) + i;
        const ulonglong2 w = W[idx];
        gs_bfly(sh[j], sh[j + (1 << lt)], w.x, w.y, q4, nq);
      }
      __syncthreads();
    }
    const u64 ni = iscale ? iscale[2 * limb].x : tb.ninv[u];
    const u64 nish = iscale ? iscale[2 * limb].y : tb.ninv_sh[u];
    for (int i = threadIdx.x; i < N; i += blockDim.x) base[i] = shoup(sh[i], ni, nish, q);
  }
}

// One-launch N = 2^16 transform on a cluster of kClusterCtas CTAs.  The row
// is the same 256 x 256 matrix as in the two-pass kernel (element h 256 + c):
// CTA q of the cluster owns columns [32 q, 32 q + 32) in the column pass and
// rows [32 q, 32 q + 32) in the row pass.  Between the passes each thread
// writes its 16 residues straight into the distributed shared memory of the
// CTA that owns them next (a column pass's residues of row h go to CTA
// h / 32), so a limb is read from and written to HBM once.  Two cluster
// barriers frame the exchange: every CTA has finished reading its own
// buffer before any is overwritten, and every write has landed before the
// second pass reads.  The butterflies, the twiddle indexing, the lazy
// ranges, the thread layouts and the ModDown epilogue are those of
// k_ntt_pass<16, 8, ..., 16, *>, so the residues are identical.
constexpr int kClusterCtas = 8;
constexpr int kMaxDevices = 64;
constexpr int kClusterThreads = 512;
constexpr int kClusterPitchA = 256 + 1;          // column pass: [32][257]
constexpr int kClusterPitchB = 256 + 256 / 16;   // row pass: [32][272], + e / 16
constexpr size_t kClusterSmem = sizeof(u64) * 32 * kClusterPitchB;

template <bool FWD, bool MD>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads, 2)
    k_ntt_cluster(u64* __restrict__ data, const RowMap rm, const NttTables tb,
                  const MdEpi epi = MdEpi{}, const ulonglong2* __restrict__ iscale = nullptr) {
  static_assert(!MD || FWD, "the ModDown epilogue ends a forward transform");
  constexpr int LOGN = 16, LS = 8, E = 16, TPS = 16, G = 32;
  extern __shared__ u64 sm[];
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int grp = (int)cluster.block_rank();  // 0..7: columns / rows 32 grp ..
  const int row = blockIdx.x / kClusterCtas;
  const int poly = row / rm.nl;
  const int limb = row - poly * rm.nl;
  const int u = rm.pidx[limb];
  u64* base = data + ((size_t)poly * rm.poly_stride + rm.off[limb]) * ((size_t)1 << LOGN);
  const u64 q = tb.mod[u].q, q4 = 4 * q, nq = 0 - q;
  const ulonglong2* W = (FWD ? tb.psi : tb.ipsi) + ((size_t)u << LOGN);
  const ulonglong2* WB = (FWD ? tb.psiB : tb.ipsiB) + (size_t)u * kTwBPerMod;
  const int t = threadIdx.x;
  // column pass: sub-transform lgA = column, thread rA of it; row pass: lgB = row
  const int lgA = t % G, rA = t / G, gA = grp * G + lgA;
  const int lgB = t / TPS, rB = t % TPS, gB = grp * G + lgB;
  auto sA = [&](int lg, int e) -> int { return lg * kClusterPitchA + e; };
  auto sB = [&](int lg, int e) -> int { return lg * kClusterPitchB + e + (e >> 4); };
  // twiddle index of the pair led by local element e at local stage sl
  auto twA = [&](int sl, int e) -> int { return (1 << sl) + (e >> (LS - sl)); };
  auto twB = [&](int sl, int e) -> int { return (1 << (8 + sl)) + (gB << sl) + (e >> (LS - sl)); };
  auto twb = [&](int sp, int m) -> ulonglong2 {  // row-pass stage sp >= 4, pair led by E rB + m
    const int off = 256 * ((1 << sp) - 16);
    return __ldg(WB + off + (gB << sp) + ((m >> (8 - sp)) << 4) + rB);
  };
  u64 x[E];
  if (FWD) {
    // ---- column pass (global stages 0-7), residues from HBM
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = base[((size_t)(rA + TPS * m) << 8) + gA];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      const int st = (E / 2) >> sp;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = __ldg(W + twA(sp, TPS * m));
        ct_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sA(lgA, rA + TPS * m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sA(lgA, E * rA + m)];
#pragma unroll
    for (int sp = 4; sp < LS; ++sp) {
      const int st = 256 >> (sp + 1);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = __ldg(W + twA(sp, E * rA + m));
        ct_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    // ---- exchange: residue h = E rA + m of column gA goes to row h's CTA
    cluster.sync();
    {
      u64* dst = cluster.map_shared_rank(sm, (unsigned)(rA >> 1));
      const int lr0 = (rA & 1) * E;
#pragma unroll
      for (int m = 0; m < E; ++m) dst[sB(lr0 + m, gA)] = x[m];
    }
    cluster.sync();
    // ---- row pass (global stages 8-15) from this CTA's buffer
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sB(lgB, rB + TPS * m)];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      const int st = (E / 2) >> sp;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = __ldg(W + twB(sp, TPS * m));
        ct_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sB(lgB, rB + TPS * m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sB(lgB, E * rB + m)];
#pragma unroll
    for (int sp = 4; sp < LS; ++sp) {
      const int st = 256 >> (sp + 1);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = twb(sp, m);
        ct_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sB(lgB, E * rB + m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = reduce_8q(sm[sB(lgB, rB + TPS * m)], q);
    if (MD) {
      // row = (item, poly p, limb) of conv [cnt][2][l][N]
      const size_t N = (size_t)1 << LOGN;
      const int item = poly >> 1, p = poly & 1;
      const u64* a = epi.acc + ((size_t)item * 2 * (epi.l + epi.K) + (size_t)p * (epi.l + epi.K) +
                                limb) * N;
      u64* o = (p ? epi.out1 : epi.out0) + item * epi.o_stride + (size_t)limb * N;
      const u64* ad = p ? epi.add1 : epi.add0;
      if (ad) ad += item * (p ? epi.a1_stride : epi.a0_stride) + (size_t)limb * N;
      const u64 pi = epi.pinv[2 * limb], pish = epi.pinv[2 * limb + 1];
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const size_t k = ((size_t)gB << 8) + rB + TPS * m;
        u64 v = shoup_est_canon(submod(a[k], x[m], q), pi, pish, q, nq);
        if (ad) v = addmod(v, ad[k], q);
        o[k] = v;
      }
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) base[((size_t)gB << 8) + rB + TPS * m] = x[m];
    }
  } else {
    // ---- row pass (global stages 15-8), residues from HBM
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = base[((size_t)gB << 8) + rB + TPS * m];
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sB(lgB, rB + TPS * m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sB(lgB, E * rB + m)];
#pragma unroll
    for (int sp = LS - 1; sp >= 4; --sp) {
      const int st = 256 >> (sp + 1);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = twb(sp, m);
        gs_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sB(lgB, E * rB + m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sB(lgB, rB + TPS * m)];
#pragma unroll
    for (int sp = 3; sp >= 0; --sp) {
      const int st = (E / 2) >> sp;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = __ldg(W + twB(sp, TPS * m));
        gs_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    // ---- exchange: residue c = rB + TPS m of row gB goes to column c's CTA
    cluster.sync();
#pragma unroll
    for (int m = 0; m < E; ++m) {
      u64* dst = cluster.map_shared_rank(sm, (unsigned)(m >> 1));
      dst[sA(rB + TPS * (m & 1), gB)] = x[m];
    }
    cluster.sync();
    // ---- column pass (global stages 7-0) from this CTA's buffer, read
    // directly in the contiguous layout of its last stages
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sA(lgA, E * rA + m)];
#pragma unroll
    for (int sp = LS - 1; sp >= 4; --sp) {
      const int st = 256 >> (sp + 1);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = __ldg(W + twA(sp, E * rA + m));
        gs_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) sm[sA(lgA, E * rA + m)] = x[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sm[sA(lgA, rA + TPS * m)];
#pragma unroll
    for (int sp = 3; sp >= 0; --sp) {
      const int st = (E / 2) >> sp;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & st) continue;
        const ulonglong2 w = __ldg(W + twA(sp, TPS * m));
        gs_bfly(x[m], x[m + st], w.x, w.y, q4, nq);
      }
    }
    const u64 ni = iscale ? iscale[2 * limb].x : tb.ninv[u];
    const u64 nish = iscale ? iscale[2 * limb].y : tb.ninv_sh[u];
#pragma unroll
    for (int m = 0; m < E; ++m) base[((size_t)(rA + TPS * m) << 8) + gA] = shoup(x[m], ni, nish, q);
  }
}

// pass A: 2^LA-point columns, pass B: 2^LB-point rows, with EA / EB residues
// per thread in NA / NB-thread CTAs, at least MB CTAs per SM
// (epi: forward only, the row pass ends with the ModDown epilogue)
template <int LOGN, int LA, int LB, int EA, int NA, int EB, int NB, int MB = 4>
static void ntt_two_pass(Context* c, u64* data, const RowMap& rm, bool fwd,
                         const MdEpi* epi = nullptr, const ulonglong2* iscale = nullptr) {
  const NttTables tb = c->tables();
  const int rows = rm.npoly * rm.nl;
  const int gA = (1 << (LOGN - LA)) / (NA / ((1 << LA) / EA));
  const int gB = (1 << (LOGN - LB)) / (NB / ((1 << LB) / EB));
  if (fwd) {
    pdl_launch(c->stream, k_ntt_pass<LOGN, LA, true, true, EA, NA, MB>, rows * gA, NA, 0, data, rm,
               tb, gA, MdEpi{}, nullptr);
    if (epi)
      pdl_launch(c->stream, k_ntt_pass<LOGN, LB, false, true, EB, NB, MB, true>, rows * gB, NB, 0,
                 data, rm, tb, gB, *epi, nullptr);
    else
      pdl_launch(c->stream, k_ntt_pass<LOGN, LB, false, true, EB, NB, MB>, rows * gB, NB, 0, data,
                 rm, tb, gB, MdEpi{}, nullptr);
  } else {
    pdl_launch(c->stream, k_ntt_pass<LOGN, LB, false, false, EB, NB, MB>, rows * gB, NB, 0, data,
               rm, tb, gB, MdEpi{}, nullptr);
    pdl_launch(c->stream, k_ntt_pass<LOGN, LA, true, false, EA, NA, MB>, rows * gA, NA, 0, data, rm,
               tb, gA, MdEpi{}, iscale);
  }
  GWHE_LAUNCHED(c, 2);
}

// the default shape of a two-pass transform: a pass of more than 8 stages
// holds 32 residues per thread in 128-thread CTAs
template <int LOGN, int LA, int LB>
static void ntt_two_pass(Context* c, u64* data, const RowMap& rm, bool fwd,
                         const MdEpi* epi = nullptr, const ulonglong2* iscale = nullptr) {
  ntt_two_pass<LOGN, LA, LB, (LA > 8 ? 32 : 16), (LA > 8 ? 128 : 256), (LB > 8 ? 32 : 16),
               (LB > 8 ? 128 : 256)>(c, data, rm, fwd, epi, iscale);
}

// the one-launch cluster transform of N = 2^16 (k_ntt_cluster)
static void ntt_cluster_16(Context* c, u64* data, const RowMap& rm, bool fwd, const MdEpi* epi,
                           const ulonglong2* iscale) {
  const NttTables tb = c->tables();
  const int rows = rm.npoly * rm.nl;
  GWHE_REQUIRE(tb.psiB && tb.ipsiB, ST_EINVAL, "row-pass twiddle table missing");
  // the kernels' dynamic shared memory above 48 KB, allowed once per device
  static std::mutex mu;
  static bool attr_set[kMaxDevices] = {};
  GWHE_REQUIRE(c->device >= 0 && c->device < kMaxDevices, ST_EINVAL, "device index out of range");
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!attr_set[c->device]) {
      GWHE_CUDA(cudaFuncSetAttribute(k_ntt_cluster<true, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterSmem));
      GWHE_CUDA(cudaFuncSetAttribute(k_ntt_cluster<true, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterSmem));
      GWHE_CUDA(cudaFuncSetAttribute(k_ntt_cluster<false, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterSmem));
      attr_set[c->device] = true;
    }
  }
  const dim3 grid((unsigned)rows * kClusterCtas);
  if (!fwd)
    k_ntt_cluster<false, false><<<grid, kClusterThreads, kClusterSmem, c->stream>>>(data, rm, tb,
                                                                                   MdEpi{}, iscale);
  else if (epi)
    k_ntt_cluster<true, true><<<grid, kClusterThreads, kClusterSmem, c->stream>>>(data, rm, tb,
                                                                                  *epi);
  else
    k_ntt_cluster<true, false><<<grid, kClusterThreads, kClusterSmem, c->stream>>>(data, rm, tb);
  GWHE_LAUNCHED(c, 1);
}

// shapes of the N = 2^16 transform (identical results; the autotuner times
// them on the device and keeps the fastest)
static void ntt_2_16(Context* c, u64* data, const RowMap& rm, bool fwd, const MdEpi* epi,
                     const ulonglong2* iscale) {
  const int rows = rm.npoly * rm.nl;
  switch (rows < kNttSmallRows ? c->ntt_variant_small : c->ntt_variant) {
    case 6: ntt_cluster_16(c, data, rm, fwd, epi, iscale); return;
    case 1: ntt_two_pass<16, 8, 8, 32, 128, 32, 128>(c, data, rm, fwd, epi, iscale); return;
    case 2: ntt_two_pass<16, 7, 9, 16, 256, 32, 128>(c, data, rm, fwd, epi, iscale); return;
    case 3: ntt_two_pass<16, 9, 7, 32, 128, 16, 256>(c, data, rm, fwd, epi, iscale); return;
    case 4: ntt_two_pass<16, 8, 8, 16, 128, 16, 128, 8>(c, data, rm, fwd, epi, iscale); return;
    case 5: ntt_two_pass<16, 8, 8, 16, 64, 16, 64, 16>(c, data, rm, fwd, epi, iscale); return;
    default: ntt_two_pass<16, 8, 8, 16, 256, 16, 256>(c, data, rm, fwd, epi, iscale); return;
  }
}

// true if the ring has a two-pass transform (and epi, if given, was applied)
static bool ntt_dispatch(Context* c, u64* data, const RowMap& rm, bool fwd,
                         const MdEpi* epi = nullptr, const ulonglong2* iscale = nullptr) {
  const int rows = rm.npoly * rm.nl;
  if (rows <= 0) return true;
  // algorithmic traffic: every residue read once and written once
  ProfScope ps(c, PROF_NTT, 16.0 * rows * c->N);
  GWHE_REQUIRE(rm.nl <= kMaxRowMap, ST_EINVAL, "too many limbs in a row map");
  switch (c->logN) {
    case 17: ntt_two_pass<17, 9, 8>(c, data, rm, fwd, epi, iscale); return true;
    case 16: ntt_2_16(c, data, rm, fwd, epi, iscale); return true;
    case 15: ntt_two_pass<15, 8, 7>(c, data, rm, fwd, epi, iscale); return true;
    case 14: ntt_two_pass<14, 7, 7>(c, data, rm, fwd, epi, iscale); return true;
    case 13: ntt_two_pass<13, 7, 6>(c, data, rm, fwd, epi, iscale); return true;
    case 12: ntt_two_pass<12, 6, 6>(c, data, rm, fwd, epi, iscale); return true;
    default: break;
  }
  if (epi) return false;
  GWHE_REQUIRE(c->logN >= 2 && c->logN <= 11, ST_EINVAL, "unsupported ring degree");
  const NttTables tb = c->tables();
  const size_t shm = sizeof(u64) << c->logN;
  if (fwd)
    pdl_launch(c->stream, k_ntt_small<true>, rows, 256, shm, data, rm, tb, c->logN, nullptr);
  else
    pdl_launch(c->stream, k_ntt_small<false>, rows, 256, shm, data, rm, tb, c->logN, iscale);
  GWHE_LAUNCHED(c, 1);
  return true;
}

void ntt_forward(Context* c, u64* data, const RowMap& rm) { ntt_dispatch(c, data, rm, true); }
bool ntt_forward_moddown(Context* c, u64* data, int cnt, const MdEpi& epi) {
  GWHE_REQUIRE(cnt >= 1 && epi.l >= 1 && epi.acc && epi.out0 && epi.out1 && epi.pinv, ST_EINVAL,
               "bad ModDown epilogue");
  if (c->logN < 12) return false;
  return ntt_dispatch(c, data, rows_q(2 * cnt, epi.l, epi.l), true, &epi);
}
void ntt_inverse(Context* c, u64* data, const RowMap& rm, const ulonglong2* iscale) {
  ntt_dispatch(c, data, rm, false, nullptr, iscale);
}

RowMap rows_q(int npoly, int l, int poly_stride) {
  GWHE_REQUIRE(l >= 0 && l <= kMaxRowLimbs, ST_EINVAL, "too many limbs");
  RowMap rm;
  rm.npoly = npoly;
  rm.nl = l;
  rm.poly_stride = poly_stride;
  for (int i = 0; i < l; ++i) {
    rm.off[i] = (uint16_t)i;
    rm.pidx[i] = (uint8_t)i;
  }
  return rm;
}

}  // namespace gwhe
