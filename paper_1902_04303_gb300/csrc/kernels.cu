// kernels.cu -- element-wise ring arithmetic, the tensor sum of the CP-REP
// product, fast base conversion (ModUp / ModDown), the key inner product,
// rescale, Galois automorphisms, ChaCha20 sampling, and the FP64 encoding
// procedure of the gwhe library.  See kernels.cuh for the interfaces.
#include <algorithm>
#include <mutex>

#include "kernels.cuh"

namespace gwhe {

namespace {

constexpr int kThreads = 256;

inline dim3 grid_rows(int N, int rows) { return dim3((N + kThreads - 1) / kThreads, rows); }

struct LimbVals {
  u64 v[kMaxRowLimbs];
  u64 sh[kMaxRowLimbs];
};

// ------------------------------------------------------------- element-wise
__global__ void k_addsub(PolyView out, CPolyView a, CPolyView b, int l, int N,
                         const DevMod* __restrict__ mod, int sub) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const u64 q = mod[i].q;
  const u64 x = a.d[((size_t)p * a.cap + i) * N + k];
  const u64 y = b.d[((size_t)p * b.cap + i) * N + k];
  out.d[((size_t)p * out.cap + i) * N + k] = sub ? submod(x, y, q) : addmod(x, y, q);
}

__global__ void k_negate(PolyView out, CPolyView a, int l, int N, const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const u64 x = a.d[((size_t)p * a.cap + i) * N + k];
  out.d[((size_t)p * out.cap + i) * N + k] = x ? mod[i].q - x : 0;
}

__global__ void k_mul_scalar(PolyView out, CPolyView a, int l, int N, const DevMod* __restrict__ mod,
                             const LimbVals v) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const u64 x = a.d[((size_t)p * a.cap + i) * N + k];
  out.d[((size_t)p * out.cap + i) * N + k] = shoup(x, v.v[i], v.sh[i], mod[i].q);
}

__global__ void k_add_scalar0(PolyView ct, int N, const DevMod* __restrict__ mod, const LimbVals v) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  u64* p = ct.d + (size_t)i * N + k;
  *p = addmod(*p, v.v[i], mod[i].q);
}

__global__ void k_mul_plain(PolyView out, CPolyView a, const u64* __restrict__ pt, int l, int N,
                            const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const u64 x = a.d[((size_t)p * a.cap + i) * N + k];
  out.d[((size_t)p * out.cap + i) * N + k] = mulmod(x, pt[(size_t)i * N + k], mod[i]);
}

__global__ void k_add_plain0(PolyView ct, const u64* __restrict__ pt, int N,
                             const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  u64* p = ct.d + (size_t)i * N + k;
  *p = addmod(*p, pt[(size_t)i * N + k], mod[i].q);
}

// ------------------------------------------------------------- base conversion
constexpr int kMaxConvIn = 16;
struct ConvArgs {
  const u64* tab;  // [n_in] hinv, [n_in] hinv_sh, [n_in][n_out] hmod
  int n_in, n_out, hm_stride, in_mod0;
  uint8_t in_pidx[kMaxConvIn];  // modulus of each input limb
  // optional constants added to every coefficient: after the input's Shoup
  // product (mod its modulus) and to each output (mod the output's modulus)
  const u64* in_add = nullptr;
  const u64* out_add = nullptr;
  // the inputs are already the products x_i hinv_i (canonical), from an
  // inverse transform scaled by the table's iscale pairs
  int pre = 0;
  uint8_t out_pidx[kMaxRowLimbs];
  uint16_t out_row[kMaxRowLimbs];
};

// y_i = [x_i hinv_i]_{m_i} (or x_i itself when the input already carries
// the factor);  out_o = sum_i y_i hmod[i][o] mod m_o.
// Grid: x = coefficients, y = groups of kConvOG outputs, z = items (polynomials).
// NI (the number of input limbs) is a template parameter, so the products and
// their 128-bit sums unroll completely; the CTA's slice of the hmod table
// (NI x kConvOG words, zero beyond the last output) is staged in shared
// memory and read as warp-uniform broadcasts.
constexpr int kConvOG = 8;
template <int NI, int T>
__device__ __forceinline__ void conv_outputs(const u64 (&y)[NI], const u64* hs, int og,
                                             int o, const ConvArgs& a, int o0, u64* op,
                                             int N, int k, const DevMod* __restrict__ mod) {
  Acc128 s[T];
#pragma unroll
  for (int t = 0; t < T; ++t) s[t] = Acc128{0, 0};
#pragma unroll
  for (int i = 0; i < NI; ++i) {
#pragma unroll
    for (int t = 0; t < T; ++t) mac128(s[t], y[i], hs[i * og + o + t]);
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int oo = o0 + o + t;
    const DevMod& om = mod[a.out_pidx[oo]];
    u64 v = reduce128(s[t].lo, s[t].hi, om);
    if (a.out_add) v = addmod(v, a.out_add[oo], om.q);
    op[(size_t)a.out_row[oo] * N + k] = v;
  }
}

// Each CTA converts one block of coefficients of one polynomial to the og
// outputs [blockIdx.y og, +og): with og = n_out (the large batches) every
// input's Shoup product is formed once per coefficient; a small batch splits
// the outputs over kConvOG-wide CTAs to fill the GPU.
template <int NI>
__global__ void __launch_bounds__(256) k_baseconv(const u64* __restrict__ x, size_t x_pstride,
                                                  u64* __restrict__ out, size_t out_pstride,
                                                  const ConvArgs a, int N, int og,
                                                  const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  __shared__ u64 hs[NI * kMaxRowLimbs];
  const int o0 = blockIdx.y * og;
  const int no = min(og, a.n_out - o0);
  for (int e = threadIdx.x; e < NI * og; e += blockDim.x) {
    const int i = e / og, o = e - i * og;
    hs[e] = o < no ? a.tab[2 * NI + i * a.hm_stride + o0 + o] : 0;
  }
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const size_t p = blockIdx.z;
  const u64* xp = x + p * x_pstride;
  u64* op = out + p * out_pstride;
  u64 y[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const u64 q = mod[a.in_pidx[i]].q;
    const u64 xv = xp[(size_t)i * N + k];
    y[i] = a.pre ? xv : shoup(xv, a.tab[i], a.tab[NI + i], q);
    if (a.in_add) y[i] = addmod(y[i], a.in_add[i], q);
  }
  int o = 0;
  for (; o + 4 <= no; o += 4) conv_outputs<NI, 4>(y, hs, og, o, a, o0, op, N, k, mod);
  switch (no - o) {
    case 3: conv_outputs<NI, 3>(y, hs, og, o, a, o0, op, N, k, mod); break;
    case 2: conv_outputs<NI, 2>(y, hs, og, o, a, o0, op, N, k, mod); break;
    case 1: conv_outputs<NI, 1>(y, hs, og, o, a, o0, op, N, k, mod); break;
    default: break;
  }
}

// Grid of the three inner-product kernels: x = groups of items, y = blocks of
// coefficients, z = extended limb u.  The groups of one (limb, coefficient
// block) are adjacent in launch order, so the key words they share are read
// from DRAM once and from L2 by the other groups.
//
// acc_p[u] = sum_j x_j[u] * key_j[p][u] over digits, for the l + K extended limbs;
// x_j[u] is the input limb itself when u lies in digit j, else the converted limb.
// Each thread keeps its key words in registers and applies them to up to IB
// items of the set, so the key is read once per IB ciphertexts.
constexpr int kKsMaxBeta = 4;
template <int IB>
// The key family has rows q_0..q_{key_lmax-1}, p_0..p_{K-1} per digit and poly.
__global__ void k_ks_inner(const u64* __restrict__ c_ntt, size_t c_stride,
                           const u64* __restrict__ ext, const u64* __restrict__ key,
                           u64* __restrict__ acc, int l, int K, int L, int key_lmax, int alpha,
                           int beta, int N, int cnt, const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int u = blockIdx.z;
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int ne = l + K;
  const int mi = u < l ? u : L + (u - l);        // modulus of extended limb u
  const int kr = u < l ? u : key_lmax + (u - l);  // its row in the key family
  const size_t KR = (size_t)(key_lmax + K);
  u64 kb[kKsMaxBeta], ka[kKsMaxBeta];
#pragma unroll
  for (int j = 0; j < kKsMaxBeta; ++j)
    if (j < beta) {
      kb[j] = key[(((size_t)j * 2 + 0) * KR + kr) * N + k];
      ka[j] = key[(((size_t)j * 2 + 1) * KR + kr) * N + k];
    }
  const DevMod m = mod[mi];
  const int it0 = blockIdx.x * IB;
  const int it1 = min(it0 + IB, cnt);
  for (int item = it0; item < it1; ++item) {
    const u64* cx = c_ntt + (size_t)item * c_stride;
    const u64* ex = ext + (size_t)item * beta * ne * N;
    Acc128 s0{0, 0}, s1{0, 0};
#pragma unroll
    for (int j = 0; j < kKsMaxBeta; ++j) {
      if (j >= beta) break;
      const int lo = j * alpha, hi = min(lo + alpha, l);
      const u64 x = (u >= lo && u < hi) ? cx[(size_t)u * N + k] : ex[((size_t)j * ne + u) * N + k];
      mac128(s0, x, kb[j]);
      mac128(s1, x, ka[j]);
    }
    u64* ac = acc + (size_t)item * 2 * ne * N;
    ac[(size_t)u * N + k] = reduce128(s0.lo, s0.hi, m);
    ac[((size_t)ne + u) * N + k] = reduce128(s1.lo, s1.hi, m);
  }
}

// NTT slot j holds a(psi^(2 brv(j) + 1)); X -> X^g maps it to slot
// brv((g (2 brv(j) + 1) mod 2N - 1) / 2) of the input.
__device__ __forceinline__ unsigned automorph_src(unsigned j, u64 g, int logN) {
  const u64 twoN_mask = ((u64)2 << logN) - 1;
  const u64 e = 2 * (u64)(__brev(j) >> (32 - logN)) + 1;
  const u64 f = (g * e) & twoN_mask;
  return __brev((unsigned)((f - 1) >> 1)) >> (32 - logN);
}

// Hoisted inner product for a sum of automorphisms: acc_p[u] = sum_g sum_j
// sigma_g(x_j)[u] * key_g,j[p][u], x_j the ModUp digits of one c1 (the input
// limb itself when u lies in digit j).  sigma_g is a permutation of NTT slots,
// applied while reading; all G beta products of an item are summed on 128
// bits (at most 28 terms below 2^120) and reduced once.  The loop runs over
// the automorphisms outside: one key's words sit in registers while they are
// applied to up to IB items, whose accumulators persist across g.
template <int IB, int G>
__global__ void k_ks_inner_hoist(const u64* __restrict__ c_ntt, size_t c_stride,
                                 const u64* __restrict__ ext, HoistKeys hk,
                                 u64* __restrict__ acc, int l, int K, int L, int key_lmax,
                                 int alpha, int beta, int logN, int cnt,
                                 const DevMod* __restrict__ mod, int accum) {
  pdl_wait();
  pdl_trigger();
  const int u = blockIdx.z;
  const int N = 1 << logN;
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int ne = l + K;
  const int mi = u < l ? u : L + (u - l);
  const int kr = u < l ? u : key_lmax + (u - l);
  const size_t KR = (size_t)(key_lmax + K);
  const int it0 = blockIdx.x * IB;
  const int nit = min(IB, cnt - it0);
  Acc128 s0[IB], s1[IB];
#pragma unroll
  for (int t = 0; t < IB; ++t) s0[t] = s1[t] = Acc128{0, 0};
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const unsigned src = automorph_src((unsigned)k, hk.g[g], logN);
    u64 kb[kKsMaxBeta], ka[kKsMaxBeta];
#pragma unroll
    for (int j = 0; j < kKsMaxBeta; ++j)
      if (j < beta) {
        kb[j] = hk.key[g][(((size_t)j * 2 + 0) * KR + kr) * N + k];
        ka[j] = hk.key[g][(((size_t)j * 2 + 1) * KR + kr) * N + k];
      }
#pragma unroll
    for (int t = 0; t < IB; ++t) {
      if (t >= nit) break;
      const int item = it0 + t;
      const u64* cx = c_ntt + (size_t)item * c_stride + (size_t)u * N;
      const u64* ex = ext + (size_t)item * beta * ne * N;
#pragma unroll
      for (int j = 0; j < kKsMaxBeta; ++j) {
        if (j >= beta) break;
        const int lo = j * alpha, hi = min(lo + alpha, l);
        const u64* row = (u >= lo && u < hi) ? cx : ex + ((size_t)j * ne + u) * N;
        const u64 x = row[src];
        mac128(s0[t], x, kb[j]);
        mac128(s1[t], x, ka[j]);
      }
    }
  }
  const DevMod m = mod[mi];
#pragma unroll
  for (int t = 0; t < IB; ++t) {
    if (t >= nit) break;
    u64* ac = acc + (size_t)(it0 + t) * 2 * ne * N;
    if (accum) {  // a later chunk of the automorphisms adds to acc
      add128(s0[t], ac[(size_t)u * N + k]);
      add128(s1[t], ac[((size_t)ne + u) * N + k]);
    }
    ac[(size_t)u * N + k] = reduce128(s0[t].lo, s0[t].hi, m);
    ac[((size_t)ne + u) * N + k] = reduce128(s1[t].lo, s1[t].hi, m);
  }
}

// The one-digit case (beta = 1: every switch at or below alpha limbs, i.e. the
// SNP batches): all G keys' words of the thread's slot stay in registers and
// the thread walks up to IB items, so each key is read once per IB items.
template <int IB, int G>
__global__ void __launch_bounds__(256, 4) k_ks_inner_hoist1(const u64* __restrict__ c_ntt,
                                                           size_t c_stride,
                                  const u64* __restrict__ ext, HoistKeys hk,
                                  u64* __restrict__ acc, int l, int K, int L, int key_lmax,
                                  int logN, int cnt, const DevMod* __restrict__ mod,
                                  int accum) {
  pdl_wait();
  pdl_trigger();
  const int u = blockIdx.z;
  const int N = 1 << logN;
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int ne = l + K;
  const int mi = u < l ? u : L + (u - l);
  const int kr = u < l ? u : key_lmax + (u - l);
  const size_t KR = (size_t)(key_lmax + K);
  unsigned src[G];
  u64 kb[G], ka[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    src[g] = automorph_src((unsigned)k, hk.g[g], logN);
    kb[g] = hk.key[g][((size_t)0 * KR + kr) * N + k];
    ka[g] = hk.key[g][((size_t)1 * KR + kr) * N + k];
  }
  const DevMod m = mod[mi];
  const int it0 = blockIdx.x * IB;
  const int it1 = min(it0 + IB, cnt);
  for (int item = it0; item < it1; ++item) {
    // digit 0 holds every limb below l: those come from c1 itself
    const u64* row = u < l ? c_ntt + (size_t)item * c_stride + (size_t)u * N
                           : ext + ((size_t)item * ne + u) * N;
    u64 x[G];
#pragma unroll
    for (int g = 0; g < G; ++g) x[g] = row[src[g]];
    u64* ac = acc + (size_t)item * 2 * ne * N;
    // a later chunk of the automorphisms adds to the earlier chunks' acc
    Acc128 s0{accum ? ac[(size_t)u * N + k] : 0, 0};
    Acc128 s1{accum ? ac[((size_t)ne + u) * N + k] : 0, 0};
#pragma unroll
    for (int g = 0; g < G; ++g) {
      mac128(s0, x[g], kb[g]);
      mac128(s1, x[g], ka[g]);
    }
    ac[(size_t)u * N + k] = reduce128(s0.lo, s0.hi, m);
    ac[((size_t)ne + u) * N + k] = reduce128(s1.lo, s1.hi, m);
  }
}

// out[item][i] = c0[item][i] + sum_g sigma_g(c0[item][i]) (NTT domain); with
// accum, out[item][i] += sum_g sigma_g(c0[item][i])
template <int G>
__global__ void k_automorph_sum(const u64* __restrict__ in, int in_cap, size_t in_stride,
                                u64* __restrict__ out, int l, int logN, HoistKeys hk,
                                const DevMod* __restrict__ mod, int accum) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.y;
  const int N = 1 << logN;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const size_t item = blockIdx.z;
  const u64* src = in + item * in_stride + (size_t)i * N;
  const u64 q = mod[i].q;
  u64* o = out + (item * l + i) * N + j;
  u64 v = accum ? *o : src[j];  // a later chunk adds to the earlier sum
#pragma unroll
  for (int g = 0; g < G; ++g) v = addmod(v, src[automorph_src((unsigned)j, hk.g[g], logN)], q);
  *o = v;
}

// out_p[i] = (acc_p[i] - conv_p[i]) P^-1 mod q_i (+ add_p[i])
__global__ void k_moddown_combine(const u64* __restrict__ acc, const u64* __restrict__ conv, int l,
                                  int K, u64* out0, u64* out1, size_t o_stride, const u64* add0,
                                  const u64* add1, size_t a0_stride, size_t a1_stride,
                                  const u64* __restrict__ pinv, int N,
                                  const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const u64 q = mod[i].q;
  const int ne = l + K;
  const size_t item = blockIdx.z;
  acc += item * (size_t)2 * ne * N;
  conv += item * (size_t)2 * l * N;
  out0 += item * o_stride;
  out1 += item * o_stride;
  if (add0) add0 += item * a0_stride;
  if (add1) add1 += item * a1_stride;
  const u64 a = acc[((size_t)p * ne + i) * N + k];
  const u64 cv = conv[((size_t)p * l + i) * N + k];
  u64 v = shoup(submod(a, cv, q), pinv[2 * i], pinv[2 * i + 1], q);
  const u64* add = p ? add1 : add0;
  if (add) v = addmod(v, add[(size_t)i * N + k], q);
  (p ? out1 : out0)[(size_t)i * N + k] = v;
}

// ------------------------------------------------------------- relin + rescale
// Fused relinearisation and rescale at level l with K special primes: the key
// product acc ([2][ne][N]) plus P (d0, d1) is divided by P' = P q_{l-1}
// through B' = {p_0..p_{K-1}, q_{l-1}}.  fz = [Pq: 2l][ppinv: 2(l-1)]
// [out_add: l-1][in_add: K+1]: P mod q_i and P'^-1 mod q_i with their Shoup
// companions, and the conversion's constants for the rounding offset
// h = floor(P'/2) added to every coefficient (in_add_j = h (P'/m_j)^-1 mod
// m_j after the input product, out_add_i = -h mod q_i on the output, which
// the combine's subtraction turns into +h).
// prep: bp[item][p][j] = y_j (NTT domain) for the B' rows
__global__ void k_fused_prep(const u64* __restrict__ acc, const u64* __restrict__ t3,
                             size_t t3_stride, int t3_cap, u64* __restrict__ bp, int l, int K,
                             int L, int N, const u64* __restrict__ fz,
                             const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, nb = K + 1, p = row / nb, j = row - p * nb;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const size_t item = blockIdx.z;
  const int ne = l + K;
  const u64* a = acc + (item * 2 + p) * (size_t)ne * N;
  u64 v;
  if (j < K) {
    v = a[(size_t)(l + j) * N + k];
  } else {
    const u64 q = mod[l - 1].q;
    const u64 d = t3[item * t3_stride + ((size_t)p * t3_cap + (l - 1)) * N + k];
    const u64 pd = shoup(d, fz[2 * (l - 1)], fz[2 * (l - 1) + 1], q);
    v = addmod(a[(size_t)(l - 1) * N + k], pd, q);
  }
  bp[((item * 2 + p) * nb + j) * (size_t)N + k] = v;
}

// combine: out_i = (acc_i + P d_i - conv_i) P'^-1 mod q_i, i < l - 1 (conv
// carries -h)
__global__ void k_fused_combine(const u64* __restrict__ acc, const u64* __restrict__ t3,
                                size_t t3_stride, int t3_cap, const u64* __restrict__ conv,
                                u64* __restrict__ out, size_t o_stride, int o_cap, int l, int K,
                                int N, const u64* __restrict__ fz,
                                const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int lo = l - 1, row = blockIdx.y, p = row / lo, i = row - p * lo;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const size_t item = blockIdx.z;
  const int ne = l + K;
  const u64 q = mod[i].q;
  const u64 a = acc[((item * 2 + p) * (size_t)ne + i) * N + k];
  const u64 d = t3[item * t3_stride + ((size_t)p * t3_cap + i) * N + k];
  const u64 cv = conv[((item * 2 + p) * (size_t)lo + i) * N + k];
  const u64* ppinv = fz + 2 * l;
  u64 y = addmod(a, shoup(d, fz[2 * i], fz[2 * i + 1], q), q);
  y = submod(y, cv, q);
  out[item * o_stride + ((size_t)p * o_cap + i) * N + k] = shoup(y, ppinv[2 * i], ppinv[2 * i + 1], q);
}

// ------------------------------------------------------------- rescale
__global__ void k_rescale_prep(const u64* __restrict__ last, int l, u64* __restrict__ tmp, int N,
                               const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, lm1 = l - 1, p = row / lm1, i = row - p * lm1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const u64 ql = mod[l - 1].q, h = ql >> 1;
  const u64 x = last[(size_t)p * N + k];
  const u64 r = (x + h >= ql) ? x + h - ql : x + h;  // (x + h) mod ql
  const DevMod m = mod[i];
  u64 v;
  if (r >= h) {
    v = reduce64(r - h, m);
  } else {
    const u64 t = reduce64(h - r, m);
    v = t ? m.q - t : 0;
  }
  tmp[((size_t)p * lm1 + i) * N + k] = v;
}

__global__ void k_rescale_combine(PolyView ct, const u64* __restrict__ tmp, int l, int N,
                                  const DevMod* __restrict__ mod, const u64* __restrict__ qlinv) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, lm1 = l - 1, p = row / lm1, i = row - p * lm1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const u64 q = mod[i].q;
  u64* c = ct.d + ((size_t)p * ct.cap + i) * N + k;
  const u64 t = tmp[((size_t)p * lm1 + i) * N + k];
  *c = shoup(submod(*c, t, q), qlinv[2 * i], qlinv[2 * i + 1], q);
}

// ------------------------------------------------------------- automorphism
// NTT slot j holds a(psi^(2 brv(j) + 1)); X -> X^g maps it to slot
// brv((g (2 brv(j) + 1) mod 2N - 1) / 2) of the input.
__global__ void k_automorph(PolyView out, CPolyView in, int l, int logN, u64 g) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int N = 1 << logN;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const u64 twoN_mask = ((u64)2 << logN) - 1;
  const u64 e = 2 * (u64)(__brev((unsigned)j) >> (32 - logN)) + 1;
  const u64 f = (g * e) & twoN_mask;
  const unsigned src = __brev((unsigned)((f - 1) >> 1)) >> (32 - logN);
  out.d[((size_t)p * out.cap + i) * N + j] = in.d[((size_t)p * in.cap + i) * N + src];
}

// ------------------------------------------------------------- ciphertext sets
// Ladder step input: out[item] = (sigma(in0) + in0, sigma(in1)) for items laid
// out at in_stride / out_stride words, cap limbs per poly.
__global__ void k_automorph_ladder(const u64* __restrict__ in, int in_cap, size_t in_stride,
                                   u64* __restrict__ out, int out_cap, size_t out_stride, int l,
                                   int logN, u64 g, const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int N = 1 << logN;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const size_t item = blockIdx.z;
  const u64* src = in + item * in_stride + ((size_t)p * in_cap + i) * N;
  const u64 twoN_mask = ((u64)2 << logN) - 1;
  const u64 e = 2 * (u64)(__brev((unsigned)j) >> (32 - logN)) + 1;
  const u64 f = (g * e) & twoN_mask;
  const unsigned srcj = __brev((unsigned)((f - 1) >> 1)) >> (32 - logN);
  u64 v = src[srcj];
  if (p == 0) v = addmod(v, src[j], mod[i].q);
  out[item * out_stride + ((size_t)p * out_cap + i) * N + j] = v;
}

// out[item] = src_item * pt_item (both polys), items listed in an array
__global__ void k_mask_set(const MaskItem* __restrict__ items, u64* __restrict__ out, int out_cap,
                           size_t out_stride, int l, int N, const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const MaskItem it = items[blockIdx.z];
  const u64 x = it.src[((size_t)p * it.src_cap + i) * N + k];
  out[blockIdx.z * out_stride + ((size_t)p * out_cap + i) * N + k] =
      mulmod(x, it.pt[(size_t)i * N + k], mod[i]);
}

// out[item] = sum over the item's npairs pairs of the tensor products
// (a0 b0, a0 b1 + a1 b0, a1 b1), on 128 bits with a reduction every 32 pairs
// (at most 64 products below 2^120 per accumulator); accumulate: out[item] +=
// that sum.  One item is the single tensor sum of the CP-REP inner loop.
__global__ void k_tensor_mac_set(PolyView out, size_t out_stride, const MacPair* __restrict__ pairs,
                                 int npairs, int l, int N, int accumulate,
                                 const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const DevMod m = mod[i];
  const size_t item = blockIdx.z;
  pairs += item * npairs;
  Acc128 s0{0, 0}, s1{0, 0}, s2{0, 0};
  const size_t off = (size_t)i * N + k;
  u64* o = out.d + item * out_stride;
  u64 r0 = 0, r1 = 0, r2 = 0;
  if (accumulate) {
    r0 = o[off];
    r1 = o[(size_t)out.cap * N + off];
    r2 = o[(size_t)2 * out.cap * N + off];
  }
  for (int j = 0; j < npairs; ++j) {
    const MacPair P = pairs[j];
    const u64 a0 = P.a[off], a1 = P.a[(size_t)P.capa * N + off];
    const u64 b0 = P.b[off], b1 = P.b[(size_t)P.capb * N + off];
    mac128(s0, a0, b0);
    mac128(s1, a0, b1);
    mac128(s1, a1, b0);
    mac128(s2, a1, b1);
    if ((j & 31) == 31) {
      r0 = addmod(r0, reduce128(s0.lo, s0.hi, m), m.q);
      r1 = addmod(r1, reduce128(s1.lo, s1.hi, m), m.q);
      r2 = addmod(r2, reduce128(s2.lo, s2.hi, m), m.q);
      s0 = Acc128{0, 0};
      s1 = Acc128{0, 0};
      s2 = Acc128{0, 0};
    }
  }
  r0 = addmod(r0, reduce128(s0.lo, s0.hi, m), m.q);
  r1 = addmod(r1, reduce128(s1.lo, s1.hi, m), m.q);
  r2 = addmod(r2, reduce128(s2.lo, s2.hi, m), m.q);
  o[off] = r0;
  o[(size_t)out.cap * N + off] = r1;
  o[(size_t)2 * out.cap * N + off] = r2;
}

// out = sum over items of the set (both polys)
__global__ void k_sum_set(const u64* __restrict__ in, int in_cap, size_t in_stride, int cnt,
                          u64* __restrict__ out, int out_cap, int l, int N,
                          const DevMod* __restrict__ mod) {
  pdl_wait();
  pdl_trigger();
  const int row = blockIdx.y, p = row / l, i = row - p * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const u64 q = mod[i].q;
  const size_t off = ((size_t)p * in_cap + i) * N + k;
  u64 acc = 0;
  for (int it = 0; it < cnt; ++it) acc = addmod(acc, in[it * in_stride + off], q);
  out[((size_t)p * out_cap + i) * N + k] = acc;
}

// ------------------------------------------------------------- ChaCha20
__device__ __forceinline__ void qround(u32& a, u32& b, u32& c, u32& d) {
  a += b; d ^= a; d = __funnelshift_l(d, d, 16);
  c += d; b ^= c; b = __funnelshift_l(b, b, 12);
  a += b; d ^= a; d = __funnelshift_l(d, d, 8);
  c += d; b ^= c; b = __funnelshift_l(b, b, 7);
}

// ChaCha20 block (RFC 8439): key words (seed lo, seed hi, 0 x 6), counter,
// nonce words (obj lo, obj hi, tag).
__device__ void chacha_block(u64 seed, u64 obj, u32 tag, u32 counter, u32 out[16]) {
  u32 s[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u, (u32)seed, (u32)(seed >> 32),
               0u, 0u, 0u, 0u, 0u, 0u, counter, (u32)obj, (u32)(obj >> 32), tag};
  u32 x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = s[i];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    qround(x[0], x[4], x[8], x[12]);
    qround(x[1], x[5], x[9], x[13]);
    qround(x[2], x[6], x[10], x[14]);
    qround(x[3], x[7], x[11], x[15]);
    qround(x[0], x[5], x[10], x[15]);
    qround(x[1], x[6], x[11], x[12]);
    qround(x[2], x[7], x[8], x[13]);
    qround(x[3], x[4], x[9], x[14]);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i] = x[i] + s[i];
}

__device__ __forceinline__ int cbd21(u32 a, u32 b) {
  return __popc(a & 0x1FFFFFu) - __popc(b & 0x1FFFFFu);
}

__device__ __forceinline__ u64 signed_to_res(i64 v, const DevMod& m) {
  if (v >= 0) return reduce64((u64)v, m);
  const u64 t = reduce64((u64)(-(v + 1)) + 1, m);
  return t ? m.q - t : 0;
}

struct PidxList {
  uint8_t u[kMaxMod];
};

// ternary: coefficient k = word k % 16 of block k / 16, value (w mod 3) - 1
__global__ void k_sample_ternary(u64 seed, u64 obj, u64* out, PidxList pl, int nl, int N,
                                 const DevMod* __restrict__ mod) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b * 16 >= N) return;
  u32 w[16];
  chacha_block(seed, obj, 0, (u32)b, w);
  for (int li = 0; li < nl; ++li) {
    const u64 q = mod[pl.u[li]].q;
    u64* o = out + (size_t)li * N + (size_t)b * 16;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int v = (int)(w[m] % 3u) - 1;
      o[m] = v < 0 ? q - 1 : (u64)v;
    }
  }
}

// centred binomial (eta 21): coefficient k = words 2(k%8), 2(k%8)+1 of block k / 8
__global__ void k_sample_cbd(u64 seed, u64 obj, u64* out, PidxList pl, int nl, int N,
                             const DevMod* __restrict__ mod) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b * 8 >= N) return;
  u32 w[16];
  chacha_block(seed, obj, 0, (u32)b, w);
  for (int li = 0; li < nl; ++li) {
    const u64 q = mod[pl.u[li]].q;
    u64* o = out + (size_t)li * N + (size_t)b * 8;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int e = cbd21(w[2 * m], w[2 * m + 1]);
      o[m] = e < 0 ? q - (u64)(-e) : (u64)e;
    }
  }
}

// uniform mod q_u: coefficient k = 128-bit word 4(k%4).. of block k / 4 of (obj, tag)
__global__ void k_sample_uniform(u64 seed, u64 obj, u32 tag, int u, u64* out, int N,
                                 const DevMod* __restrict__ mod) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b * 4 >= N) return;
  u32 w[16];
  chacha_block(seed, obj, tag, (u32)b, w);
  const DevMod m = mod[u];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const u64 lo = (u64)w[4 * r] | ((u64)w[4 * r + 1] << 32);
    const u64 hi = (u64)w[4 * r + 2] | ((u64)w[4 * r + 3] << 32);
    out[(size_t)b * 4 + r] = reduce128(lo, hi, m);
  }
}

// encryption randomness for ct idx (enc id id0 + idx): a CTA of 256 threads
// covers 4096 coefficients; each thread draws the ChaCha20 blocks of its 16
// coefficients into shared memory, then the residues are written coalesced.
__global__ void __launch_bounds__(256) k_enc_sample(u64 seed, u64 id0, const u64* __restrict__ ids,
                                                    int count, int l,
                                                    const i64* __restrict__ m_coeff,
                                                    u64* __restrict__ tmp, int N,
                                                    const DevMod* __restrict__ mod) {
  __shared__ int8_t sv[4096], se1[4096];
  __shared__ i64 sme[4096];
  const int tiles = (N + 4095) / 4096;
  const int idx = blockIdx.x / tiles;
  const int tile = blockIdx.x - idx * tiles;
  if (idx >= count) return;
  const int base = tile * 4096;
  const int tcoef = min(4096, N - base);
  const u64 id = ids ? ids[idx] : id0 + (u64)idx;
  const int tid = threadIdx.x;
  if (tid * 16 < tcoef) {
    const int b = (base >> 4) + tid;  // ternary block of coefficients 16b..16b+15
    u32 wv[16], wa[16], wb[16];
    chacha_block(seed, (3ull << 48) | id, 0, (u32)b, wv);
#pragma unroll
    for (int m = 0; m < 16; ++m) sv[tid * 16 + m] = (int8_t)((int)(wv[m] % 3u) - 1);
    chacha_block(seed, (4ull << 48) | id, 0, (u32)(2 * b), wa);
    chacha_block(seed, (4ull << 48) | id, 0, (u32)(2 * b + 1), wb);
    const i64* mc = m_coeff + (size_t)idx * N + base + tid * 16;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      sme[tid * 16 + m] = mc[m] + (i64)cbd21(wa[2 * m], wa[2 * m + 1]);
      sme[tid * 16 + 8 + m] = mc[8 + m] + (i64)cbd21(wb[2 * m], wb[2 * m + 1]);
    }
    chacha_block(seed, (5ull << 48) | id, 0, (u32)(2 * b), wa);
    chacha_block(seed, (5ull << 48) | id, 0, (u32)(2 * b + 1), wb);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      se1[tid * 16 + m] = (int8_t)cbd21(wa[2 * m], wa[2 * m + 1]);
      se1[tid * 16 + 8 + m] = (int8_t)cbd21(wb[2 * m], wb[2 * m + 1]);
    }
  }
  __syncthreads();
  u64* t = tmp + (size_t)idx * 3 * l * N + base;
  for (int i = 0; i < l; ++i) {
    const DevMod md = mod[i];
    u64* t0 = t + (size_t)i * N;
    u64* t1 = t + ((size_t)l + i) * N;
    u64* t2 = t + ((size_t)2 * l + i) * N;
    for (int k = tid; k < tcoef; k += 256) {
      const int v = sv[k], e1 = se1[k];
      t0[k] = v < 0 ? md.q - 1 : (u64)v;
      t1[k] = signed_to_res(sme[k], md);
      t2[k] = e1 < 0 ? md.q - (u64)(-e1) : (u64)e1;
    }
  }
}

// c0 = v b + t0, c1 = v a + t1 (NTT domain), pk = [2][L][N]
__global__ void k_enc_combine(const u64* __restrict__ tmp, int l, const u64* __restrict__ pk,
                              int L, u64* __restrict__ out, int out_cap, size_t out_stride, int N,
                              const DevMod* __restrict__ mod) {
  const int row = blockIdx.y, idx = row / l, i = row - idx * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const DevMod m = mod[i];
  const u64* t = tmp + (size_t)idx * 3 * l * N;
  const u64 v = t[(size_t)i * N + k];
  const u64 t0 = t[((size_t)l + i) * N + k];
  const u64 t1 = t[((size_t)2 * l + i) * N + k];
  const u64 b = pk[(size_t)i * N + k];
  const u64 a = pk[((size_t)L + i) * N + k];
  u64* o = out + idx * out_stride;
  o[(size_t)i * N + k] = addmod(mulmod(v, b, m), t0, m.q);
  o[((size_t)out_cap + i) * N + k] = addmod(mulmod(v, a, m), t1, m.q);
}

__global__ void k_ksk_combine(u64* b, const u64* __restrict__ a, const u64* __restrict__ e,
                              const u64* __restrict__ s, const u64* __restrict__ t, u64 pmod, int u,
                              int N, const DevMod* __restrict__ mod) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const DevMod m = mod[u];
  u64 v = submod(e[k], mulmod(a[k], s[k], m), m.q);
  if (t) v = addmod(v, mulmod(pmod, t[k], m), m.q);
  b[k] = v;
}

__global__ void k_int_to_rns(const i64* __restrict__ in, int count, int l, u64* __restrict__ out,
                             int N, const DevMod* __restrict__ mod) {
  const int row = blockIdx.y, idx = row / l, i = row - idx * l;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  out[((size_t)idx * l + i) * N + k] = signed_to_res(in[(size_t)idx * N + k], mod[i]);
}

__global__ void k_decrypt(CPolyView ct, const u64* __restrict__ s, int l, u64* __restrict__ m,
                          int N, const DevMod* __restrict__ mod) {
  const int i = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const DevMod md = mod[i];
  const u64 c0 = ct.d[(size_t)i * N + k];
  const u64 c1 = ct.d[((size_t)ct.cap + i) * N + k];
  m[(size_t)i * N + k] = addmod(c0, mulmod(c1, s[(size_t)i * N + k], md), md.q);
}

// m[i] = c0_i + c1_i s on the q0 limb (NTT domain) for a list of ciphertexts
__global__ void k_decrypt_q0_list(const u64* const* __restrict__ c0s,
                                  const u64* const* __restrict__ c1s,
                                  const u64* __restrict__ s, u64* __restrict__ m, int N,
                                  const DevMod* __restrict__ mod) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const size_t i = blockIdx.y;
  const DevMod md = mod[0];
  m[i * N + k] = addmod(c0s[i][k], mulmod(c1s[i][k], s[k], md), md.q);
}

__global__ void k_gather_slots(const double2* __restrict__ z, int cnt, int M, int B, int stride,
                               double2* __restrict__ out) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)cnt * B) return;
  const long i = t / B, b = t - i * B;
  out[t] = z[i * M + b * stride];
}

// ------------------------------------------------------------- encoding FFT
// Complex arithmetic as separately rounded IEEE operations (no FMA), in the
// order of the encoding procedure.
__device__ __forceinline__ double2 cmul_exact(double2 a, double2 b) {
  return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                      __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ void fft_bfly(double2& x, double2& y, double2 w) {
  const double2 t = cmul_exact(y, w);
  const double2 a = x;
  x = make_double2(__dadd_rn(a.x, t.x), __dadd_rn(a.y, t.y));
  y = make_double2(__dsub_rn(a.x, t.x), __dsub_rn(a.y, t.y));
}

// radix-2 stages len = 2 .. 2^a inside tiles of 2^a contiguous entries
__global__ void k_fft_tile(double2* __restrict__ G, const double2* __restrict__ W, int logM, int a) {
  extern __shared__ double2 sf[];
  const int T = 1 << a;
  const int M = 1 << logM;
  double2* base = G + (size_t)blockIdx.x * T;
  for (int i = threadIdx.x; i < T; i += blockDim.x) sf[i] = base[i];
  __syncthreads();
  for (int ls = 1; ls <= a; ++ls) {
    const int half = 1 << (ls - 1);
    const int stride = M >> ls;
    for (int b = threadIdx.x; b < (T >> 1); b += blockDim.x) {
      const int blk = b >> (ls - 1), jj = b & (half - 1);
      const int p = (blk << ls) + jj;
      fft_bfly(sf[p], sf[p + half], W[jj * stride]);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < T; i += blockDim.x) base[i] = sf[i];
}

// remaining stages len = 2^(a+1) .. M: thread per (transform, low index lo),
// R = M / 2^a entries in registers
template <int R>
__global__ void k_fft_cols(double2* __restrict__ G, const double2* __restrict__ W, int logM, int a,
                           int count) {
  const int T = 1 << a, M = 1 << logM;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)count * T) return;
  const size_t idx = gid / T;
  const int lo = (int)(gid - idx * T);
  double2* base = G + idx * M;
  double2 x[R];
#pragma unroll
  for (int h = 0; h < R; ++h) x[h] = base[(size_t)h * T + lo];
#pragma unroll
  for (int s2 = 0; (1 << s2) < R; ++s2) {
    const int hs = 1 << s2;
    const int stride = M >> (a + 1 + s2);
#pragma unroll
    for (int h = 0; h < R; ++h) {
      if (h & hs) continue;
      const int jj = ((h & (hs - 1)) << a) + lo;
      fft_bfly(x[h], x[h + hs], W[jj * stride]);
    }
  }
#pragma unroll
  for (int h = 0; h < R; ++h) base[(size_t)h * T + lo] = x[h];
}

// ------------------------------------------------------------- fixed-point encoding
// The encoding procedure in exact integer arithmetic (the same statement as
// the library header): values are int64 fixed-point with F = 61 - log2 M - e
// fractional bits, twiddles carry 62 fractional bits, every complex product is
// formed on 128 bits and rounded as (v + 2^61) >> 62.
// (p1 - p2 + 2^61) >> 62 for exact signed 128-bit products p1 = a1 b1, p2 =
// a2 b2, sign +1 (or p1 + p2 for sign -1), from 64-bit low/high halves; the
// result fits in 64 bits.
__device__ __forceinline__ i64 fx_dot(i64 a1, i64 b1, i64 a2, i64 b2, bool sub) {
  const u64 l1 = (u64)a1 * (u64)b1, l2 = (u64)a2 * (u64)b2;
  const i64 h1 = __mul64hi(a1, b1), h2 = __mul64hi(a2, b2);
  u64 lo;
  i64 hi;
  if (sub) {
    lo = l1 - l2;
    hi = h1 - h2 - (l1 < l2 ? 1 : 0);
  } else {
    lo = l1 + l2;
    hi = h1 + h2 + (lo < l1 ? 1 : 0);
  }
  const u64 r = lo + ((u64)1 << 61);
  hi += (r < lo ? 1 : 0);
  return (i64)(((u64)hi << 2) | (r >> 62));
}
__device__ __forceinline__ longlong2 cmul_fx(longlong2 a, longlong2 w) {
  return make_longlong2(fx_dot(a.x, w.x, a.y, w.y, true), fx_dot(a.x, w.y, a.y, w.x, false));
}
__device__ __forceinline__ void fx_bfly(longlong2& x, longlong2& y, longlong2 w) {
  const longlong2 t = cmul_fx(y, w);
  const longlong2 a = x;
  x = make_longlong2(a.x + t.x, a.y + t.y);
  y = make_longlong2(a.x - t.x, a.y - t.y);
}

// e[idx] = smallest e in [0, 40] with 2^e >= max |Re|, |Im| of plaintext idx.
// Pass 1: per block, the maximum magnitude as the bit pattern of a
// non-negative double (ordered like the value), atomically maxed per plaintext.
__global__ void k_enc_maxabs(const double2* __restrict__ z, int M, int blocks_per,
                             unsigned long long* __restrict__ mx) {
  __shared__ double red[256];
  const int idx = blockIdx.x / blocks_per, part = blockIdx.x - idx * blocks_per;
  const int chunk = (M + blocks_per - 1) / blocks_per;
  const double2* zz = z + (size_t)idx * M;
  double m = 0.0;
  for (int j = part * chunk + threadIdx.x; j < min(M, (part + 1) * chunk); j += blockDim.x) {
    const double2 v = zz[j];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(mx + idx, (unsigned long long)__double_as_longlong(red[0]));
}
// pass 2: the exponent from the maximum
__global__ void k_enc_exponent(const unsigned long long* __restrict__ mx, int count,
                               int* __restrict__ e) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const double m = __longlong_as_double((long long)mx[idx]);
  int ex = 0;
  while (ex < 40 && scalbn(1.0, ex) < m) ++ex;
  e[idx] = ex;
}

// Twist and round one entry k of transform idx: c = G Tq[k], coefficient
// k = rint((double)Re c * f), k + M = rint((double)Im c * f).
__device__ __forceinline__ void fx_emit(longlong2 g, const longlong2* __restrict__ T, int k,
                                        int M, double f, i64* o) {
  const longlong2 c = cmul_fx(g, T[k]);
  o[k] = __double2ll_rn(__dmul_rn(__ll2double_rn(c.x), f));
  o[k + M] = __double2ll_rn(__dmul_rn(__ll2double_rn(c.y), f));
}

// Radix-2 stages len = 2 .. 2^a inside tiles of 2^a contiguous entries of the
// bit-reversed input: entry p of transform idx is loaded as the fixed-point
// value of slot inv[p] (F = 61 - logM - e[idx]).  When the tile is the whole
// transform (a = logM) the twist and rounding are applied here.
__global__ void k_fx_tile(const double2* __restrict__ z, const int* __restrict__ inv,
                          const int* __restrict__ e, longlong2* __restrict__ G,
                          const longlong2* __restrict__ W, const longlong2* __restrict__ Tq,
                          int logM, int a, double scale, i64* __restrict__ out) {
  extern __shared__ longlong2 sfx[];
  const int T = 1 << a;
  const int M = 1 << logM;
  const int tiles = M >> a;
  const size_t idx = blockIdx.x / tiles;
  const int t0 = (blockIdx.x - (int)(idx * tiles)) * T;
  const int F = 61 - logM - e[idx];
  const double2* zz = z + idx * M;
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    const double2 v = zz[inv[t0 + i]];
    sfx[i] = make_longlong2(__double2ll_rn(scalbn(v.x, F)), __double2ll_rn(scalbn(v.y, F)));
  }
  __syncthreads();
  for (int ls = 1; ls <= a; ++ls) {
    const int half = 1 << (ls - 1);
    const int stride = M >> ls;
    for (int b = threadIdx.x; b < (T >> 1); b += blockDim.x) {
      const int blk = b >> (ls - 1), jj = b & (half - 1);
      const int p = (blk << ls) + jj;
      fx_bfly(sfx[p], sfx[p + half], W[jj * stride]);
    }
    __syncthreads();
  }
  if (a == logM) {
    const double f = scalbn(scale, -(logM + F));
    i64* o = out + idx * 2 * M;
    for (int i = threadIdx.x; i < T; i += blockDim.x) fx_emit(sfx[i], Tq, i, M, f, o);
  } else {
    longlong2* base = G + idx * M + t0;
    for (int i = threadIdx.x; i < T; i += blockDim.x) base[i] = sfx[i];
  }
}

// remaining stages len = 2^(a+1) .. M, R entries per thread in registers,
// then the twist and rounding of those R entries
template <int R>
__global__ void k_fx_cols(const longlong2* __restrict__ G, const longlong2* __restrict__ W,
                          const longlong2* __restrict__ Tq, const int* __restrict__ e, int logM,
                          int a, int count, double scale, i64* __restrict__ out) {
  const int T = 1 << a, M = 1 << logM;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)count * T) return;
  const size_t idx = gid / T;
  const int lo = (int)(gid - idx * T);
  const longlong2* base = G + idx * M;
  longlong2 x[R];
#pragma unroll
  for (int h = 0; h < R; ++h) x[h] = base[(size_t)h * T + lo];
#pragma unroll
  for (int s2 = 0; (1 << s2) < R; ++s2) {
    const int hs = 1 << s2;
    const int stride = M >> (a + 1 + s2);
#pragma unroll
    for (int h = 0; h < R; ++h) {
      if (h & hs) continue;
      const int jj = ((h & (hs - 1)) << a) + lo;
      fx_bfly(x[h], x[h + hs], W[jj * stride]);
    }
  }
  const int F = 61 - logM - e[idx];
  const double f = scalbn(scale, -(logM + F));
  i64* o = out + idx * 2 * M;
#pragma unroll
  for (int h = 0; h < R; ++h) fx_emit(x[h], Tq, h * T + lo, M, f, o);
}

// decoding: centred residues mod q0 -> (m_k + i m_(k+M)) T[k] at bit-reversed k
__global__ void k_decode_prep(const u64* __restrict__ m, const double2* __restrict__ T, int logM,
                              int count, u64 q, double2* __restrict__ G) {
  const int M = 1 << logM;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)count * M) return;
  const size_t idx = gid / M;
  const int k = (int)(gid - idx * M);
  const u64* mp = m + idx * 2 * M;
  const u64 a = mp[k], b = mp[k + M];
  const double re = a > q / 2 ? -(double)(q - a) : (double)a;
  const double im = b > q / 2 ? -(double)(q - b) : (double)b;
  const int p = (int)(__brev((unsigned)k) >> (32 - logM));
  G[idx * M + p] = cmul_exact(make_double2(re, im), T[k]);
}

__global__ void k_decode_gather(const double2* __restrict__ G, const int* __restrict__ u, int M,
                                int count, double scale, double2* __restrict__ z) {
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)count * M) return;
  const size_t idx = gid / M;
  const int j = (int)(gid - idx * M);
  const double2 g = G[idx * M + u[j]];
  z[gid] = make_double2(g.x / scale, g.y / scale);
}

// S holds the genotype columns [col0, col0 + width) of every sample, row pitch ld
__global__ void k_build_snp_rep(const double* __restrict__ S, long ld, long col0, int n, long k,
                                long k0, int nb, int B, int M, double2* __restrict__ z) {
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)n * M) return;
  const size_t j = gid / M;
  const int s = (int)(gid - j * M);
  const int b = s / nb;
  const long col = k0 + 2L * b;
  double re = 0.0, im = 0.0;
  if (b < B) {
    if (col < k) re = S[j * (size_t)ld + (col - col0)];
    if (col + 1 < k) im = S[j * (size_t)ld + (col + 1 - col0)];
  }
  z[gid] = make_double2(re, im);
}

// CCP SNP batches (factored layout): batch i of count, slot b*nb + t =
// S[t, c] + i S[t, c + 1] with c = k0 + i*tau + 2b, zero for t >= n or c >= k
__global__ void k_build_snp_ccp(const double* __restrict__ S, long ld, long col0, int n, long k,
                                long k0, int count,
                                int tau, int nb, int B, int M, double2* __restrict__ z) {
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)count * M) return;
  const size_t i = gid / M;
  const int s = (int)(gid - i * M);
  const int b = s / nb, t = s - b * nb;
  const long col = k0 + (long)i * tau + 2L * b;
  double re = 0.0, im = 0.0;
  if (b < B && t < n) {
    if (col < k) re = S[(size_t)t * ld + (col - col0)];
    if (col + 1 < k) im = S[(size_t)t * ld + (col + 1 - col0)];
  }
  z[gid] = make_double2(re, im);
}

inline unsigned blocks_for(size_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ============================================================= wrappers
void ew_addsub(Context* c, PolyView out, CPolyView a, CPolyView b, int npoly, int l, bool sub) {
  ProfScope ps(c, PROF_ELEMWISE, 3.0 * npoly * l * 8.0 * c->N);
  if (npoly * l == 0) return;
  pdl_launch(c->stream, k_addsub, grid_rows(c->N, npoly * l), kThreads, 0, out, a, b, l, c->N,
             c->d_mod, sub ? 1 : 0);
  GWHE_LAUNCHED(c, 1);
}

void ew_negate(Context* c, PolyView out, CPolyView a, int npoly, int l) {
  ProfScope ps(c, PROF_ELEMWISE, 2.0 * npoly * l * 8.0 * c->N);
  if (npoly * l == 0) return;
  pdl_launch(c->stream, k_negate, grid_rows(c->N, npoly * l), kThreads, 0, out, a, l, c->N,
             c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

static LimbVals make_vals(Context* c, int l, const u64* v) {
  GWHE_REQUIRE(l <= kMaxRowLimbs, ST_EINVAL, "too many limbs");
  LimbVals lv;
  for (int i = 0; i < l; ++i) {
    lv.v[i] = v[i] % c->mod[i];
    lv.sh[i] = shoup_companion(lv.v[i], c->mod[i]);
  }
  return lv;
}

void ew_mul_scalar(Context* c, PolyView out, CPolyView a, int npoly, int l, const u64* v) {
  ProfScope ps(c, PROF_ELEMWISE, 2.0 * npoly * l * 8.0 * c->N);
  if (npoly * l == 0) return;
  pdl_launch(c->stream, k_mul_scalar, grid_rows(c->N, npoly * l), kThreads, 0, out, a, l, c->N,
             c->d_mod, make_vals(c, l, v));
  GWHE_LAUNCHED(c, 1);
}

void ew_add_scalar_poly0(Context* c, PolyView ct, int l, const u64* v) {
  ProfScope ps(c, PROF_ELEMWISE, 2.0 * l * 8.0 * c->N);
  if (l == 0) return;
  pdl_launch(c->stream, k_add_scalar0, grid_rows(c->N, l), kThreads, 0, ct, c->N, c->d_mod,
             make_vals(c, l, v));
  GWHE_LAUNCHED(c, 1);
}

void ew_mul_plain(Context* c, PolyView out, CPolyView a, int npoly, int l, const u64* pt) {
  ProfScope ps(c, PROF_ELEMWISE, (2.0 * npoly + 1) * l * 8.0 * c->N);
  if (npoly * l == 0) return;
  pdl_launch(c->stream, k_mul_plain, grid_rows(c->N, npoly * l), kThreads, 0, out, a, pt, l, c->N,
             c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void ew_add_plain_poly0(Context* c, PolyView ct, int l, const u64* pt) {
  ProfScope ps(c, PROF_ELEMWISE, 3.0 * l * 8.0 * c->N);
  if (l == 0) return;
  pdl_launch(c->stream, k_add_plain0, grid_rows(c->N, l), kThreads, 0, ct, pt, c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

static ConvArgs conv_args(const ConvTable& t, int in_mod0) {
  GWHE_REQUIRE(t.n_in <= kMaxConvIn && t.n_out <= kMaxRowLimbs, ST_EINVAL, "conversion too large");
  ConvArgs a;
  a.tab = t.dev;
  a.n_in = t.n_in;
  a.n_out = t.n_out;
  a.hm_stride = t.n_out;
  a.in_mod0 = in_mod0;
  for (int i = 0; i < t.n_in; ++i)
    a.in_pidx[i] = (uint8_t)(t.in_pidx.empty() ? in_mod0 + i : t.in_pidx[i]);
  for (int o = 0; o < t.n_out; ++o) {
    a.out_pidx[o] = t.out_pidx[o];
    a.out_row[o] = t.out_limb[o];
  }
  return a;
}

static void launch_baseconv(Context* c, const u64* x, size_t xs, u64* out, size_t os, int cnt,
                            const ConvArgs& a) {
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "conversion batch too large");
  GWHE_REQUIRE(a.n_out >= 1 && a.n_out <= kMaxRowLimbs, ST_EINVAL, "conversion outputs");
  // all outputs per CTA once the launch has at least two waves of CTAs
  // (152 SMs x 8 CTAs of 256 threads), else kConvOG outputs per CTA
  const long ctas = (long)blocks_for(c->N) * cnt;
  const int og = ctas >= 2L * 152 * 8 ? a.n_out : std::min(a.n_out, kConvOG);
  const dim3 grid(blocks_for(c->N), (a.n_out + og - 1) / og, cnt);
#define GWHE_CONV_CASE(n)                                                                      \
  case n:                                                                                      \
    pdl_launch(c->stream, k_baseconv<n>, grid, kThreads, 0, x, xs, out, os, a, c->N, og,        \
               c->d_mod);                                                                      \
    break;
  switch (a.n_in) {
    GWHE_CONV_CASE(1) GWHE_CONV_CASE(2) GWHE_CONV_CASE(3) GWHE_CONV_CASE(4)
    GWHE_CONV_CASE(5) GWHE_CONV_CASE(6) GWHE_CONV_CASE(7) GWHE_CONV_CASE(8)
    GWHE_CONV_CASE(9) GWHE_CONV_CASE(10) GWHE_CONV_CASE(11) GWHE_CONV_CASE(12)
    GWHE_CONV_CASE(13) GWHE_CONV_CASE(14) GWHE_CONV_CASE(15) GWHE_CONV_CASE(16)
    default: GWHE_REQUIRE(false, ST_EINVAL, "conversion input count out of range");
  }
#undef GWHE_CONV_CASE
  GWHE_LAUNCHED(c, 1);
}

void modup_convert_set(Context* c, const u64* x_coeff, int l, u64* ext, int cnt, bool pre) {
  ProfScope ps(c, PROF_BASECONV, 0.0);
  const int beta = (l + c->alpha - 1) / c->alpha;
  const int ne = l + c->ks_k[l];
  const size_t N = c->N;
  for (int j = 0; j < beta; ++j) {
    const ConvTable& t = c->modup.at({l, j});
    ConvArgs a = conv_args(t, t.in_lo);
    a.pre = pre;
    ps.bytes += 8.0 * (t.n_in + t.n_out) * N * cnt;
    launch_baseconv(c, x_coeff + (size_t)t.in_lo * N, (size_t)l * N, ext + (size_t)j * ne * N,
                    (size_t)beta * ne * N, cnt, a);
  }
}

void moddown_convert_set(Context* c, const u64* acc, int l, int K, u64* conv, int cnt, bool pre) {
  GWHE_REQUIRE(l >= 1 && l <= c->P.L && K >= 1 && K <= c->P.K && c->d_pinv[K], ST_EINVAL,
               "bad level or special-prime count");
  ProfScope ps(c, PROF_BASECONV, 2.0 * cnt * (K + l) * 8.0 * c->N);
  const int ne = l + K;
  ConvArgs a = conv_args(c->moddown[K], c->P.L);  // table rows hold all L outputs
  a.n_out = l;                                    // produce the first l of them
  a.pre = pre;
  // items: the 2 cnt polynomials of acc ([cnt][2][ne][N]) -> conv ([cnt][2][l][N])
  launch_baseconv(c, acc + (size_t)l * c->N, (size_t)ne * c->N, conv, (size_t)l * c->N, 2 * cnt, a);
}

void moddown_combine_set(Context* c, const u64* acc, const u64* conv, int l, int K, int cnt,
                         u64* out0, u64* out1, size_t o_stride, const u64* add0, const u64* add1,
                         size_t a0_stride, size_t a1_stride) {
  ProfScope ps(c, PROF_ELEMWISE, 2.0 * 3 * l * cnt * 8.0 * c->N);
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "batch too large");
  pdl_launch(c->stream, k_moddown_combine, dim3(blocks_for(c->N), 2 * l, cnt), kThreads, 0, acc,
             conv, l, K, out0, out1, o_stride, add0, add1, a0_stride, a1_stride, c->d_pinv[K], c->N,
             c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void ks_inner_set(Context* c, const u64* c_ntt, size_t c_stride, int l, const u64* ext,
                  const Ksk& key, u64* acc, int cnt) {
  const int K = key.k;
  const double ne_ = l + K, beta_ = (l + c->alpha - 1) / c->alpha;
  ProfScope ps(c, PROF_KS_INNER, (3.0 * beta_ * ne_ + 2.0 * ne_) * 8.0 * c->N * cnt);
  const int beta = (l + c->alpha - 1) / c->alpha;
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "batch too large");
  GWHE_REQUIRE(beta <= kKsMaxBeta, ST_EINVAL, "more than 4 key digits at one level");
  GWHE_REQUIRE(key.d && key.lmax >= l && beta <= key.dk, ST_ENOKEY, "key family does not reach the level");
  constexpr int IB = 8;
  pdl_launch(c->stream, k_ks_inner<IB>, dim3((cnt + IB - 1) / IB, blocks_for(c->N), l + K),
             kThreads, 0, c_ntt, c_stride, ext, key.d, acc, l, K, c->P.L, key.lmax, c->alpha, beta,
             c->N, cnt, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

template <int G>
static void launch_hoist(Context* c, const u64* c_ntt, size_t c_stride, int l, const u64* ext,
                         const HoistKeys& hk, int key_lmax, int K, u64* acc, int cnt, int beta,
                         int accum) {
  if (beta == 1) {
    constexpr int IB1 = 32;
    const dim3 grid((cnt + IB1 - 1) / IB1, blocks_for(c->N), l + K);
    pdl_launch(c->stream, k_ks_inner_hoist1<IB1, G>, grid, kThreads, 0, c_ntt, c_stride, ext, hk,
               acc, l, K, c->P.L, key_lmax, c->logN, cnt, c->d_mod, accum);
    return;
  }
  // items per thread (each key word is read once per IB items): eight with up
  // to three automorphisms; with more, one.  The multi-digit kernel is bound
  // by the latency of its key reads and gathers, and one item per thread (46
  // registers, five CTAs per SM) measured faster than four or five per thread
  // (72-80 registers, three CTAs per SM), though each key word is then read
  // once per item; the grid puts a limb's items next to each other in launch
  // order, so those reads after the first come from L2
  constexpr int IB = G <= 3 ? 8 : 1;
  const dim3 grid((cnt + IB - 1) / IB, blocks_for(c->N), l + K);
  pdl_launch(c->stream, k_ks_inner_hoist<IB, G>, grid, kThreads, 0, c_ntt, c_stride, ext, hk, acc,
             l, K, c->P.L, key_lmax, c->alpha, beta, c->logN, cnt, c->d_mod, accum);
}

void ks_inner_hoist_set(Context* c, const u64* c_ntt, size_t c_stride, int l, const u64* ext,
                        const HoistKeys& hk, int key_lmax, int K, u64* acc, int cnt) {
  const double ne_ = l + K, beta_ = (l + c->alpha - 1) / c->alpha;
  ProfScope ps(c, PROF_KS_INNER, ((1.0 + 2.0 * hk.G) * beta_ * ne_ + 2.0 * ne_) * 8.0 * c->N * cnt);
  const int beta = (l + c->alpha - 1) / c->alpha;
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "batch too large");
  GWHE_REQUIRE(beta <= kKsMaxBeta, ST_EINVAL, "more than 4 key digits at one level");
  GWHE_REQUIRE(hk.G >= 1 && hk.G <= kMaxHoist, ST_EINVAL, "bad hoisted automorphism count");
  // chunks of up to kHoistChunk automorphisms; each later chunk adds its
  // products to acc (exact sums mod each modulus, so the chunking does not
  // change the result)
  for (int g0 = 0; g0 < hk.G; g0 += kHoistChunk) {
    HoistKeys part;
    part.G = std::min(kHoistChunk, hk.G - g0);
    for (int g = 0; g < part.G; ++g) {
      part.key[g] = hk.key[g0 + g];
      part.g[g] = hk.g[g0 + g];
    }
    const int accum = g0 > 0;
    switch (part.G) {
#define GWHE_HOIST(n)                                                                             \
  case n:                                                                                         \
    launch_hoist<n>(c, c_ntt, c_stride, l, ext, part, key_lmax, K, acc, cnt, beta, accum);        \
    break;
      GWHE_HOIST(1) GWHE_HOIST(2) GWHE_HOIST(3) GWHE_HOIST(4) GWHE_HOIST(5) GWHE_HOIST(6)
      GWHE_HOIST(7)
#undef GWHE_HOIST
      default: throw Error(ST_EINVAL, "hoisted chunk out of range");
    }
    GWHE_LAUNCHED(c, 1);
  }
}

void automorph_sum_set(Context* c, const u64* in, int in_cap, size_t in_stride, u64* out, int l,
                       int cnt, const HoistKeys& hk) {
  ProfScope ps(c, PROF_ELEMWISE, (1.0 + hk.G) * l * cnt * 8.0 * c->N);
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "batch too large");
  GWHE_REQUIRE(hk.G >= 1 && hk.G <= kMaxHoist, ST_EINVAL, "bad hoisted automorphism count");
  const dim3 grid(blocks_for(c->N), l, cnt);
  for (int g0 = 0; g0 < hk.G; g0 += kHoistChunk) {
    HoistKeys part;
    part.G = std::min(kHoistChunk, hk.G - g0);
    for (int g = 0; g < part.G; ++g) {
      part.key[g] = hk.key[g0 + g];
      part.g[g] = hk.g[g0 + g];
    }
    const int accum = g0 > 0;
#define GWHE_AUTOSUM(G)                                                                          \
  case G:                                                                                        \
    pdl_launch(c->stream, k_automorph_sum<G>, grid, kThreads, 0, in, in_cap, in_stride, out, l,  \
               c->logN, part, c->d_mod, accum);                                                  \
    break;
    switch (part.G) {
      GWHE_AUTOSUM(1) GWHE_AUTOSUM(2) GWHE_AUTOSUM(3) GWHE_AUTOSUM(4) GWHE_AUTOSUM(5)
      GWHE_AUTOSUM(6) GWHE_AUTOSUM(7)
      default: throw Error(ST_EINVAL, "hoisted chunk out of range");
    }
#undef GWHE_AUTOSUM
    GWHE_LAUNCHED(c, 1);
  }
}

void fused_prep_set(Context* c, const u64* acc, const u64* t3, size_t t3_stride, int t3_cap,
                    u64* bp, int l, int K, int cnt) {
  ProfScope ps(c, PROF_ELEMWISE, 3.0 * 2 * (K + 1) * cnt * 8.0 * c->N);
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536 && l >= 2, ST_EINVAL, "bad fused batch");
  pdl_launch(c->stream, k_fused_prep, dim3(blocks_for(c->N), 2 * (K + 1), cnt), kThreads, 0, acc,
             t3, t3_stride, t3_cap, bp, l, K, c->P.L, c->N, c->d_fused[l], c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void fused_convert_set(Context* c, const u64* bp, int l, int K, u64* conv, int cnt, bool pre) {
  ProfScope ps(c, PROF_BASECONV, 2.0 * cnt * (K + l) * 8.0 * c->N);
  const ConvTable& t = c->fused[l];
  GWHE_REQUIRE(t.n_in == K + 1 && t.n_out == l - 1, ST_EINVAL, "fused conversion table");
  ConvArgs a = conv_args(t, 0);
  a.out_add = c->d_fused[l] + 2 * l + 2 * (l - 1);
  a.in_add = a.out_add + (l - 1);
  a.pre = pre;
  launch_baseconv(c, bp, (size_t)(K + 1) * c->N, conv, (size_t)(l - 1) * c->N, 2 * cnt, a);
}

void fused_combine_set(Context* c, const u64* acc, const u64* t3, size_t t3_stride, int t3_cap,
                       const u64* conv, u64* out, size_t o_stride, int o_cap, int l, int K,
                       int cnt) {
  ProfScope ps(c, PROF_ELEMWISE, 4.0 * 2 * (l - 1) * cnt * 8.0 * c->N);
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536 && l >= 2, ST_EINVAL, "bad fused batch");
  pdl_launch(c->stream, k_fused_combine, dim3(blocks_for(c->N), 2 * (l - 1), cnt), kThreads, 0, acc,
             t3, t3_stride, t3_cap, conv, out, o_stride, o_cap, l, K, c->N, c->d_fused[l],
             c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void automorph_ladder_set(Context* c, const u64* in, int in_cap, size_t in_stride, u64* out,
                          int out_cap, size_t out_stride, int l, int cnt, u64 g) {
  ProfScope ps(c, PROF_ELEMWISE, 2.0 * 2 * l * cnt * 8.0 * c->N);
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "batch too large");
  pdl_launch(c->stream, k_automorph_ladder, dim3(blocks_for(c->N), 2 * l, cnt), kThreads, 0, in,
             in_cap, in_stride, out, out_cap, out_stride, l, c->logN, g, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void mask_set(Context* c, const MaskItem* d_items, int cnt, u64* out, int out_cap,
              size_t out_stride, int l) {
  ProfScope ps(c, PROF_ELEMWISE, 5.0 * l * cnt * 8.0 * c->N);
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "batch too large");
  pdl_launch(c->stream, k_mask_set, dim3(blocks_for(c->N), 2 * l, cnt), kThreads, 0, d_items, out,
             out_cap, out_stride, l, c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void tensor_mac_set(Context* c, PolyView out3, size_t out_stride, const MacPair* d_pairs,
                    int npairs, int cnt, int l, bool accumulate) {
  ProfScope ps(c, PROF_TENSOR_MAC, (4.0 * npairs + 3.0) * l * cnt * 8.0 * c->N);
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "batch too large");
  pdl_launch(c->stream, k_tensor_mac_set, dim3(blocks_for(c->N), l, cnt), kThreads, 0, out3,
             out_stride, d_pairs, npairs, l, c->N, accumulate ? 1 : 0, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void sum_set(Context* c, const u64* in, int in_cap, size_t in_stride, int cnt, u64* out,
             int out_cap, int l) {
  ProfScope ps(c, PROF_ELEMWISE, (2.0 * cnt + 2.0) * l * 8.0 * c->N);
  pdl_launch(c->stream, k_sum_set, dim3(blocks_for(c->N), 2 * l), kThreads, 0, in, in_cap,
             in_stride, cnt, out, out_cap, l, c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void rescale_prep(Context* c, const u64* last, int npoly, int l, u64* tmp) {
  ProfScope ps(c, PROF_ELEMWISE, (npoly + npoly * (l - 1.0)) * 8.0 * c->N);
  pdl_launch(c->stream, k_rescale_prep, grid_rows(c->N, npoly * (l - 1)), kThreads, 0, last, l, tmp,
             c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void rescale_combine(Context* c, PolyView ct, const u64* tmp_ntt, int npoly, int l) {
  ProfScope ps(c, PROF_ELEMWISE, 3.0 * npoly * (l - 1.0) * 8.0 * c->N);
  const u64* qlinv = c->d_rescale + (size_t)l * c->P.L * 2;
  pdl_launch(c->stream, k_rescale_combine, grid_rows(c->N, npoly * (l - 1)), kThreads, 0, ct,
             tmp_ntt, l, c->N, c->d_mod, qlinv);
  GWHE_LAUNCHED(c, 1);
}

void automorph_ntt(Context* c, PolyView out, CPolyView in, int npoly, int l, u64 g) {
  ProfScope ps(c, PROF_ELEMWISE, 2.0 * npoly * l * 8.0 * c->N);
  if (npoly * l == 0) return;
  pdl_launch(c->stream, k_automorph, grid_rows(c->N, npoly * l), kThreads, 0, out, in, l, c->logN,
             g);
  GWHE_LAUNCHED(c, 1);
}

static PidxList make_pl(const uint8_t* pidx, int nl) {
  GWHE_REQUIRE(nl <= kMaxMod, ST_EINVAL, "too many limbs");
  PidxList pl;
  for (int i = 0; i < nl; ++i) pl.u[i] = pidx[i];
  return pl;
}

void sample_ternary_rns(Context* c, u64 obj, u64* out, const uint8_t* pidx, int nl) {
  ProfScope ps(c, PROF_SAMPLE, 1.0 * nl * 8.0 * c->N);
  k_sample_ternary<<<blocks_for(c->N / 16), kThreads, 0, c->stream>>>(
      c->seed, obj, out, make_pl(pidx, nl), nl, c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void sample_cbd_rns(Context* c, u64 obj, u64* out, const uint8_t* pidx, int nl) {
  ProfScope ps(c, PROF_SAMPLE, 1.0 * nl * 8.0 * c->N);
  k_sample_cbd<<<blocks_for(c->N / 8), kThreads, 0, c->stream>>>(c->seed, obj, out,
                                                                 make_pl(pidx, nl), nl, c->N,
                                                                 c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void sample_uniform(Context* c, u64 obj, u32 tag, int u, u64* out) {
  ProfScope ps(c, PROF_SAMPLE, 8.0 * c->N);
  k_sample_uniform<<<blocks_for(c->N / 4), kThreads, 0, c->stream>>>(c->seed, obj, tag, u, out,
                                                                     c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void enc_sample(Context* c, u64 id0, int count, int l, const i64* m_coeff, u64* tmp,
                const u64* d_ids) {
  ProfScope ps(c, PROF_SAMPLE, (3.0 * l + 1.0) * count * 8.0 * c->N);
  if (count == 0) return;
  const int tiles = (c->N + 4095) / 4096;
  k_enc_sample<<<(unsigned)((size_t)count * tiles), 256, 0, c->stream>>>(
      c->seed, id0, d_ids, count, l, m_coeff, tmp, c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void enc_combine(Context* c, const u64* tmp_ntt, int count, int l, u64* out, int out_cap,
                 size_t out_stride) {
  ProfScope ps(c, PROF_SAMPLE, 5.0 * count * l * 8.0 * c->N);
  if (count == 0) return;
  GWHE_REQUIRE((size_t)count * l < 65536, ST_EINVAL, "encryption batch too large");
  k_enc_combine<<<grid_rows(c->N, count * l), kThreads, 0, c->stream>>>(
      tmp_ntt, l, c->d_pk, c->P.L, out, out_cap, out_stride, c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void ksk_combine(Context* c, u64* b, const u64* a, const u64* e, const u64* s, const u64* t,
                 u64 pmod, int u) {
  ProfScope ps(c, PROF_ELEMWISE, 5.0 * 8.0 * c->N);
  k_ksk_combine<<<blocks_for(c->N), kThreads, 0, c->stream>>>(b, a, e, s, t, pmod, u, c->N,
                                                             c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void int_to_rns(Context* c, const i64* in, int count, int l, u64* out) {
  ProfScope ps(c, PROF_ELEMWISE, (1.0 + l) * count * 8.0 * c->N);
  if (count * l == 0) return;
  GWHE_REQUIRE((size_t)count * l < 65536, ST_EINVAL, "batch too large");
  k_int_to_rns<<<grid_rows(c->N, count * l), kThreads, 0, c->stream>>>(in, count, l, out, c->N,
                                                                       c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void decrypt_q0_list(Context* c, const u64* const* d_c0s, const u64* const* d_c1s, int cnt,
                     u64* m) {
  ProfScope ps(c, PROF_ELEMWISE, 4.0 * cnt * 8.0 * c->N);
  GWHE_REQUIRE(cnt >= 1 && cnt < 65536, ST_EINVAL, "decryption batch too large");
  k_decrypt_q0_list<<<dim3(blocks_for(c->N), cnt), kThreads, 0, c->stream>>>(d_c0s, d_c1s, c->d_sk, m,
                                                                           c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

void gather_slots(Context* c, const double2* z, int cnt, int M, int B, int stride, double2* out) {
  GWHE_REQUIRE(cnt >= 1 && B >= 1 && stride >= 1 && (long)(B - 1) * stride < M, ST_EINVAL,
               "slot gather out of range");
  const long n = (long)cnt * B;
  k_gather_slots<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(z, cnt, M, B,
                                                                                     stride, out);
  GWHE_LAUNCHED(c, 1);
}

void decrypt_ntt(Context* c, CPolyView ct, int l, u64* m) {
  ProfScope ps(c, PROF_ELEMWISE, 4.0 * l * 8.0 * c->N);
  k_decrypt<<<grid_rows(c->N, l), kThreads, 0, c->stream>>>(ct, c->d_sk, l, m, c->N, c->d_mod);
  GWHE_LAUNCHED(c, 1);
}

static void fft_stages(Context* c, double2* G, const double2* W, int count) {
  const int logM = c->logN - 1, M = 1 << logM;
  const int a = logM < 12 ? logM : 12;  // 4096-entry tiles: 64 KiB of shared memory
  const int T = 1 << a;
  static std::once_flag smem_opt_in;
  std::call_once(smem_opt_in, [] {
    GWHE_CUDA(cudaFuncSetAttribute(k_fft_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(double2) * 4096));
  });
  k_fft_tile<<<(unsigned)((size_t)count * (M / T)), 256, sizeof(double2) * T, c->stream>>>(G, W,
                                                                                          logM, a);
  GWHE_LAUNCHED(c, 1);
  const int R = M / T;
  const unsigned nb = blocks_for((size_t)count * T, 128);
  switch (R) {
    case 1: break;
    case 2: k_fft_cols<2><<<nb, 128, 0, c->stream>>>(G, W, logM, a, count); break;
    case 4: k_fft_cols<4><<<nb, 128, 0, c->stream>>>(G, W, logM, a, count); break;
    case 8: k_fft_cols<8><<<nb, 128, 0, c->stream>>>(G, W, logM, a, count); break;
    case 16: k_fft_cols<16><<<nb, 128, 0, c->stream>>>(G, W, logM, a, count); break;
    default: throw Error(ST_EINVAL, "ring degree too large for the encoder");
  }
  GWHE_LAUNCHED(c, 1);
}

void encode_batch(Context* c, const double2* z, int count, double scale, i64* out, double2* work) {
  ProfScope ps(c, PROF_ENCODE, 2.0 * count * 16.0 * (c->N / 2));
  if (count == 0) return;
  const int logM = c->logN - 1, M = 1 << logM;
  const int a = logM < 12 ? logM : 12;  // 4096-entry tiles: 64 KiB of shared memory
  const int T = 1 << a;
  // opt in to 64 KiB of dynamic shared memory once per process (idempotent,
  // safe from several threads)
  static std::once_flag smem_opt_in;
  std::call_once(smem_opt_in, [] {
    GWHE_CUDA(cudaFuncSetAttribute(k_fx_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(longlong2) * 4096));
  });
  longlong2* G = (longlong2*)work;  // same size as count * M double2
  int* e = (int*)dalloc_bytes(c, (sizeof(int) + sizeof(unsigned long long)) * count + 8);
  unsigned long long* mx = (unsigned long long*)(e + count + (count & 1));
  GWHE_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * count, c->stream));
  const int blocks_per = M >= 8192 ? 16 : 1;
  k_enc_maxabs<<<count * blocks_per, 256, 0, c->stream>>>(z, M, blocks_per, mx);
  k_enc_exponent<<<blocks_for(count), kThreads, 0, c->stream>>>(mx, count, e);
  k_fx_tile<<<(unsigned)((size_t)count * (M / T)), 256, sizeof(longlong2) * T, c->stream>>>(
      z, c->d_slot_inv, e, G, c->d_fftWq, c->d_fftTq, logM, a, scale, out);
  const int R = M / T;
  const unsigned nb = blocks_for((size_t)count * T, 128);
  switch (R) {
    case 1: break;
    case 2: k_fx_cols<2><<<nb, 128, 0, c->stream>>>(G, c->d_fftWq, c->d_fftTq, e, logM, a, count, scale, out); break;
    case 4: k_fx_cols<4><<<nb, 128, 0, c->stream>>>(G, c->d_fftWq, c->d_fftTq, e, logM, a, count, scale, out); break;
    case 8: k_fx_cols<8><<<nb, 128, 0, c->stream>>>(G, c->d_fftWq, c->d_fftTq, e, logM, a, count, scale, out); break;
    case 16: k_fx_cols<16><<<nb, 128, 0, c->stream>>>(G, c->d_fftWq, c->d_fftTq, e, logM, a, count, scale, out); break;
    default: throw Error(ST_EINVAL, "ring degree too large for the encoder");
  }
  dfree(c, e);
  GWHE_LAUNCHED(c, R > 1 ? 4 : 3);
}

void decode_batch(Context* c, const u64* m_coeff_q0, int count, double scale, double2* z,
                  double2* work) {
  ProfScope ps(c, PROF_ENCODE, 2.0 * count * 16.0 * (c->N / 2));
  if (count == 0) return;
  const int logM = c->logN - 1, M = 1 << logM;
  k_decode_prep<<<blocks_for((size_t)count * M), kThreads, 0, c->stream>>>(
      m_coeff_q0, c->d_fftT_dec, logM, count, c->mod[0], work);
  GWHE_LAUNCHED(c, 1);
  fft_stages(c, work, c->d_fftW_dec, count);
  k_decode_gather<<<blocks_for((size_t)count * M), kThreads, 0, c->stream>>>(work, c->d_slot_u, M,
                                                                            count, scale, z);
  GWHE_LAUNCHED(c, 1);
}

void build_snp_rep(Context* c, const double* S, long ld, long col0, int n, long k, long k0, int nb,
                   int B, int M, double2* z) {
  ProfScope ps(c, PROF_ELEMWISE, 16.0 * n * M);
  GWHE_REQUIRE(k0 >= col0 && ld >= 1, ST_EINVAL, "genotype columns not held");
  k_build_snp_rep<<<blocks_for((size_t)n * M), kThreads, 0, c->stream>>>(S, ld, col0, n, k, k0, nb,
                                                                          B, M, z);
  GWHE_LAUNCHED(c, 1);
}

void build_snp_ccp(Context* c, const double* S, long ld, long col0, int n, long k, long k0,
                   int count, int tau, int nb, int B, int M, double2* z) {
  ProfScope ps(c, PROF_ELEMWISE, 16.0 * (double)count * M);
  if (count == 0) return;
  GWHE_REQUIRE(k0 >= col0 && ld >= 1, ST_EINVAL, "genotype columns not held");
  k_build_snp_ccp<<<blocks_for((size_t)count * M), kThreads, 0, c->stream>>>(
      S, ld, col0, n, k, k0, count, tau, nb, B, M, z);
  GWHE_LAUNCHED(c, 1);
}

}  // namespace gwhe
