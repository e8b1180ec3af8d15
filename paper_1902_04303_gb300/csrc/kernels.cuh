// kernels.cuh -- launch wrappers of the element-wise, base-conversion,
// sampling and encoding kernels (kernels.cu).  All work is enqueued on the
// context's stream; buffers are device pointers.
#pragma once

#include "core.cuh"

namespace gwhe {

// A set of polynomials over the q-limbs: poly p, limb i at d + (p * cap + i) * N.
struct PolyView {
  u64* d;
  int cap;
};
struct CPolyView {
  const u64* d;
  int cap;
};

// One term of a tensor sum: ciphertexts a, b (2 polys each).
struct MacPair {
  const u64* a;
  const u64* b;
  int capa, capb;
};

// One item of a batched mask product: out = src (2 polys, src_cap) * pt.
struct MaskItem {
  const u64* src;
  int src_cap;
  const u64* pt;
};

// element-wise (NTT or coefficient domain; limb i is modulo q_i)
void ew_addsub(Context* c, PolyView out, CPolyView a, CPolyView b, int npoly, int l, bool sub);
void ew_negate(Context* c, PolyView out, CPolyView a, int npoly, int l);
// out = a * v_i for limb i (v[i] < q_i)
void ew_mul_scalar(Context* c, PolyView out, CPolyView a, int npoly, int l, const u64* v);
// c0 limb i += v[i] in every coefficient (a constant polynomial in the NTT domain)
void ew_add_scalar_poly0(Context* c, PolyView ct, int l, const u64* v);
// out_p = a_p * pt for p < npoly
void ew_mul_plain(Context* c, PolyView out, CPolyView a, int npoly, int l, const u64* pt);
// c0 += pt
void ew_add_plain_poly0(Context* c, PolyView ct, int l, const u64* pt);

// key switching pieces, over cnt items (strides in words).  A switch at level
// l uses K = ks_k[l] special primes; ext rows: for each digit j, ne = l + K
// limbs at ext + (j * ne + u) * N.
// pre: the inputs already carry the conversion's hinv factor (inverse
// transform with the table's iscale pairs)
void modup_convert_set(Context* c, const u64* x_coeff, int l, u64* ext, int cnt, bool pre = false);
void moddown_convert_set(Context* c, const u64* acc, int l, int K, u64* conv, int cnt,
                         bool pre = false);
void ks_inner_set(Context* c, const u64* c_ntt, size_t c_stride, int l, const u64* ext,
                  const Ksk& key, u64* acc, int cnt);
void moddown_combine_set(Context* c, const u64* acc, const u64* conv, int l, int K, int cnt,
                         u64* out0, u64* out1, size_t o_stride, const u64* add0, const u64* add1,
                         size_t a0_stride, size_t a1_stride);
// Relinearisation fused with rescale (level l, K = ks_k[l] special primes),
// over cnt tensors (t3 items at t3 + i t3_stride, cap t3_cap): bp rows
// [cnt][2][K+1][N] of y + floor(P'/2) over B' = {p_0..p_{K-1}, q_{l-1}},
// their conversion to q_0..q_{l-2} ([cnt][2][l-1][N]), and the combine.
void fused_prep_set(Context* c, const u64* acc, const u64* t3, size_t t3_stride, int t3_cap,
                    u64* bp, int l, int K, int cnt);
void fused_convert_set(Context* c, const u64* bp, int l, int K, u64* conv, int cnt,
                       bool pre = false);
void fused_combine_set(Context* c, const u64* acc, const u64* t3, size_t t3_stride, int t3_cap,
                       const u64* conv, u64* out, size_t o_stride, int o_cap, int l, int K,
                       int cnt);
// Hoisted key switching of a sum of automorphisms (at most kMaxHoist): the
// Galois elements and the key family each uses.
constexpr int kMaxHoist = 15;
// automorphisms per inner-product launch (the kernels keep a chunk's keys in
// registers); longer sums run in chunks that accumulate
constexpr int kHoistChunk = 7;
struct HoistKeys {
  const u64* key[kMaxHoist];
  u64 g[kMaxHoist];
  int G;
};
// acc = sum_g <sigma_g(ModUp digits), key_g> for cnt items (c_ntt: the items' c1)
void ks_inner_hoist_set(Context* c, const u64* c_ntt, size_t c_stride, int l, const u64* ext,
                        const HoistKeys& hk, int key_lmax, int K, u64* acc, int cnt);
// out[item] ([cnt][l][N]) = c0 + sum_g sigma_g(c0), c0 = item poly 0
void automorph_sum_set(Context* c, const u64* in, int in_cap, size_t in_stride, u64* out, int l,
                       int cnt, const HoistKeys& hk);
// out[item] = (sigma_g(in0) + in0, sigma_g(in1)): the automorphism of a ladder step
void automorph_ladder_set(Context* c, const u64* in, int in_cap, size_t in_stride, u64* out,
                          int out_cap, size_t out_stride, int l, int cnt, u64 g);
void mask_set(Context* c, const MaskItem* d_items, int cnt, u64* out, int out_cap,
              size_t out_stride, int l);
void tensor_mac_set(Context* c, PolyView out3, size_t out_stride, const MacPair* d_pairs,
                    int npairs, int cnt, int l, bool accumulate = false);
void sum_set(Context* c, const u64* in, int in_cap, size_t in_stride, int cnt, u64* out,
             int out_cap, int l);

// rescale pieces: last = coefficient-domain last limbs [npoly][N]
void rescale_prep(Context* c, const u64* last, int npoly, int l, u64* tmp);
void rescale_combine(Context* c, PolyView ct, const u64* tmp_ntt, int npoly, int l);

// Galois automorphism X -> X^g applied to NTT-domain limbs
void automorph_ntt(Context* c, PolyView out, CPolyView in, int npoly, int l, u64 g);

// sampling (ChaCha20, see the library header for the stream layout)
void sample_ternary_rns(Context* c, u64 obj, u64* out, const uint8_t* pidx, int nl);
void sample_cbd_rns(Context* c, u64 obj, u64* out, const uint8_t* pidx, int nl);
void sample_uniform(Context* c, u64 obj, u32 tag, int u, u64* out);
// batched encryption randomness: for ct idx < count (enc id = id0 + idx):
// tmp[idx][0] = v, tmp[idx][1] = m + e0, tmp[idx][2] = e1 over l q-limbs;
// with d_ids (device array) the enc id of ct idx is d_ids[idx]
void enc_sample(Context* c, u64 id0, int count, int l, const i64* m_coeff, u64* tmp,
                const u64* d_ids = nullptr);
void enc_combine(Context* c, const u64* tmp_ntt, int count, int l, u64* out, int out_cap,
                 size_t out_stride);
// key-switching key limb: b = -a s + e (+ Pt)
void ksk_combine(Context* c, u64* b, const u64* a, const u64* e, const u64* s, const u64* t,
                 u64 pmod, int u);

// encoding procedure (see params / library header) and decoding
void encode_batch(Context* c, const double2* z, int count, double scale, i64* out, double2* work);
void int_to_rns(Context* c, const i64* in, int count, int l, u64* out);
void decode_batch(Context* c, const u64* m_coeff_q0, int count, double scale, double2* z,
                  double2* work);

// decryption inner product m = c0 + c1 s over l limbs (NTT domain)
// m[i] = c0_i + c1_i s on limb 0 (NTT domain) for cnt ciphertexts given by
// device arrays of their poly pointers
void decrypt_q0_list(Context* c, const u64* const* d_c0s, const u64* const* d_c1s, int cnt,
                     u64* m);
// out[i * B + b] = z[i * M + b * stride] for i < cnt, b < B: the slots of a
// batch of decoded vectors that hold results, gathered before the copy back
void gather_slots(Context* c, const double2* z, int cnt, int M, int B, int stride, double2* out);
void decrypt_ntt(Context* c, CPolyView ct, int l, u64* m);

// The genotype source of both builders is a device array holding the columns
// col0.. of every sample's row, row pitch ld: genotype S[j, col] is at
// S[j * ld + col - col0] (the whole n x k matrix: ld = k, col0 = 0).
// REP rows of a SNP batch as complex slots: rows j < n, slot b * nb + t =
// S[j, k0 + 2b] + i S[j, k0 + 2b + 1] (zero beyond k)
void build_snp_rep(Context* c, const double* S, long ld, long col0, int n, long k, long k0, int nb,
                   int B, int M, double2* z);
// count CCP SNP batches from k0 (tau SNPs each): slot b*nb + t of batch i =
// S[t, k0 + i tau + 2b] + i S[t, k0 + i tau + 2b + 1]
void build_snp_ccp(Context* c, const double* S, long ld, long col0, int n, long k, long k0,
                   int count, int tau, int nb, int B, int M, double2* z);

}  // namespace gwhe
