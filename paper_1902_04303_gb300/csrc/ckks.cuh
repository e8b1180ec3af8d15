// ckks.cuh -- RNS-CKKS context, keys and evaluator of the gwhe library
// (scheme of the paper's section "Homomorphic Encryption": KeyGen, Encrypt,
// Decrypt, Add, Mult, Rescale, Encode/Decode, Rotate, in RNS form with hybrid
// key switching).
#pragma once

#include <tuple>
#include <utility>
#include <vector>

#include "kernels.cuh"

namespace gwhe {

// random-stream object ids (nonce words 0-1 of the ChaCha20 stream)
constexpr u64 kObjSk = 1;
constexpr u64 kObjPkA = 2;
constexpr u64 kObjPkE = 3;
inline u64 obj_ksk_a(u32 key, int k, int j) {
  return (1ull << 40) | ((u64)k << 32) | ((u64)key << 8) | (u64)j;
}
inline u64 obj_ksk_e(u32 key, int k, int j) {
  return (2ull << 40) | ((u64)k << 32) | ((u64)key << 8) | (u64)j;
}

Context* ctx_create(const Params& P, u64 seed, cudaStream_t stream);
void ctx_destroy(Context* c);
// a context on another stream sharing base's tables and keys (base must
// outlive it and hold its keys; no key generation on the child)
Context* ctx_child(const Context* base, cudaStream_t stream);

void keygen(Context* c, const std::vector<u32>& galois);
void add_galois_key(Context* c, u32 g);
u32 galois_for_rotation(const Context* c, int r);
u32 galois_conj(const Context* c);

CtPtr ct_new(Context* c, int npoly, int cap, int l, double scale);
CtPtr ct_clone(Context* c, const Ct& a);

// arithmetic (all on the context's stream)
void op_addsub(Context* c, const Ct& a, const Ct& b, Ct& out, bool sub);
void op_negate(Context* c, const Ct& a, Ct& out);
void op_add_const(Context* c, Ct& ct, double v);
void op_mul_int(Context* c, Ct& ct, i64 k);
void op_mul_const(Context* c, Ct& ct, double v);
void op_mul_plain(Context* c, const Ct& a, const u64* pt, double pt_scale, Ct& out);
void op_add_plain(Context* c, Ct& ct, const u64* pt);
void op_tensor_mac(Context* c, const std::vector<std::pair<const Ct*, const Ct*>>& terms, Ct& out3);
void op_relin(Context* c, const Ct& t3, Ct& out);
void op_rescale(Context* c, Ct& ct);
void op_mult(Context* c, const Ct& a, const Ct& b, Ct& out);
void op_galois(Context* c, const Ct& a, u32 g, Ct& out);
void op_rotate(Context* c, const Ct& a, int r, Ct& out);
void op_conj(Context* c, const Ct& a, Ct& out);
void op_drop(Ct& ct, int l);

// key switch of the NTT-domain l-limb polynomial x: out_p = KS(x)_p (+ add_p)
void keyswitch(Context* c, const u64* x_ntt, int l, const KeySet& key, u64* out0, u64* out1,
               const u64* add0, const u64* add1);

// encoding: z (device, count x M complex) -> plaintexts (device, NTT domain,
// count x l limbs, contiguous)
void encode_to_ntt(Context* c, const double2* z, int count, double scale, int l, u64* pt);
// a public slot vector from the host, cached by (kind, index, level, scale)
const u64* mask_pt(Context* c, int kind, long index, int l, double scale,
                   const std::vector<double2>& slots);
// batched encryption of count plaintext slot vectors (device) into
// ciphertexts [count][2][out_cap][N] (level l <= out_cap); enc id of ct idx =
// id0 + idx
void encrypt_slots(Context* c, const double2* z, int count, double scale, int l, u64 id0,
                   u64* out, int out_cap, const u64* d_ids = nullptr);
void encrypt_coeffs(Context* c, const i64* m, int count, int l, u64 id0, u64* out, int out_cap,
                    const u64* d_ids = nullptr);

// host transfers in the coefficient domain
void ct_import(Context* c, Ct& ct, const u64* host_coeff, int npoly, int l, double scale);
void ct_export(Context* c, const Ct& ct, u64* host_coeff);
void decrypt_coeff(Context* c, const Ct& ct, u64* dev_out);  // [l][N] coefficient domain

// A set of cnt ciphertexts (npoly polys each, room for cap limbs) in one
// allocation: item i, poly p, limb k at d + ((i * npoly + p) * cap + k) * N.
// All items share a level and a scale.  Independent ciphertexts of the
// circuit (the columns of M, the entries being replicated, the SNP batches)
// are processed as one set so that every kernel launch covers all of them.
struct CtSet {
  Context* ctx = nullptr;
  u64* d = nullptr;
  int cnt = 0, npoly = 2, cap = 0, l = 0;
  double scale = 1.0;
  bool owned = true;
  bool is_output = false;  // holds a job's kept batch results
  ~CtSet();
  // non-owning set over items [first, first + n) at level lv (lv <= l)
  CtSet slice(int first, int n, int lv) const;
  size_t stride() const { return (size_t)npoly * cap * ctx->N; }
  u64* item(int i) const { return d + (size_t)i * stride(); }
  CtPtr view(int i) const;  // non-owning ciphertext of item i
  Ct all() const;           // the whole set as one npoly*cnt-poly ciphertext (non-owning)
};
typedef std::unique_ptr<CtSet> CtSetPtr;
CtSetPtr set_new(Context* c, int cnt, int npoly, int cap, int l, double scale);

// batched key switch: item i reads x + i x_stride (l limbs, NTT domain) and
// writes out0/out1 + i o_stride (+ add0 + i a0_stride, add1 + i a1_stride)
void keyswitch_set(Context* c, const u64* x, size_t x_stride, int cnt, int l, const KeySet& key,
                   u64* out0, u64* out1, size_t o_stride, const u64* add0, const u64* add1,
                   size_t a0_stride, size_t a1_stride);
// s[i] += Rotate(s[i], step) for each step in turn (Alg. 1/4/5/7 ladders),
// evaluated as hoisted sums over the groups of ladder_groups(steps, group).
// Up to `group` consecutive doubling steps (r, 2r, 4r, ...) -> one group
// {r, 2r, ..., (2^group - 1) r}; a shorter run of m -> {r, .., (2^m - 1) r}.
// Every ladder of the circuit takes groups of kLadderGroup steps: at the SNP
// batch levels one ModUp and ModDown of a ciphertext costs about as much as
// eleven automorphisms' inner products and sums, which makes three steps (7
// rotations) per group the fastest split of an 8-step ladder (four steps,
// 15 rotations, measured slower).
constexpr int kLadderGroup = 3;
void set_ladder(Context* c, CtSet& s, const std::vector<int>& steps, int group = kLadderGroup);
// s[i] += sum_{r in rs} Rotate(s[i], r) with the key switches hoisted (one
// ModUp, one ModDown; at most kMaxHoist = 15 rotations)
void set_rotate_sum(Context* c, CtSet& s, const std::vector<int>& rs);
std::vector<std::vector<int>> ladder_groups(const std::vector<int>& steps,
                                            int group = kLadderGroup);
// out[i] = automorphism g of a[i] (rotation or conjugation)
void set_galois(Context* c, const CtSet& a, u32 g, CtSet& out);
// out[i] = items[i].src * items[i].pt, scale = src scale * pt_scale (then rescale)
void set_mask(Context* c, const std::vector<MaskItem>& items, double src_scale, double pt_scale,
              CtSet& out, bool rescale);
// out3[i] = sum_j tensor(pairs[i npairs + j]) (out3 has npoly = 3); with
// accumulate, out3[i] += that sum (out3 already at the pairs' level and scale)
void set_tensor_mac(Context* c, const std::vector<std::pair<const Ct*, const Ct*>>& pairs,
                    int npairs, CtSet& out3, bool accumulate = false);
void set_relin(Context* c, const CtSet& t3, CtSet& out);
// relinearisation fused with the rescale that follows it: out = the tensor
// divided once by P q_{l-1} (level l - 1, scale / q_{l-1})
void set_relin_rescale(Context* c, const CtSet& t3, CtSet& out);
void op_relin_rescale(Context* c, const Ct& t3, Ct& out);
void set_rescale(Context* c, CtSet& s);
// out[i] = a_i * b_i (tensor, relinearise, rescale)
void set_mult(Context* c, const std::vector<std::pair<const Ct*, const Ct*>>& pairs, CtSet& out);

// pool allocation of temporaries: freed at scope exit (stream-ordered)
struct Tmp {
  Context* c;
  void* p;
  Tmp(Context* c_, size_t bytes);
  ~Tmp();
  u64* u() const { return (u64*)p; }
  template <class T>
  T* as() const {
    return (T*)p;
  }
};

}  // namespace gwhe
