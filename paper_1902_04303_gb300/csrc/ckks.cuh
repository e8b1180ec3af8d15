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
inline u64 obj_ksk_a(u32 key, int j) { return (1ull << 40) | ((u64)key << 8) | (u64)j; }
inline u64 obj_ksk_e(u32 key, int j) { return (2ull << 40) | ((u64)key << 8) | (u64)j; }

Context* ctx_create(const Params& P, u64 seed, cudaStream_t stream);
void ctx_destroy(Context* c);

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
void keyswitch(Context* c, const u64* x_ntt, int l, const Ksk& key, u64* out0, u64* out1,
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
                   u64* out, int out_cap);
void encrypt_coeffs(Context* c, const i64* m, int count, int l, u64 id0, u64* out, int out_cap);

// host transfers in the coefficient domain
void ct_import(Context* c, Ct& ct, const u64* host_coeff, int npoly, int l, double scale);
void ct_export(Context* c, const Ct& ct, u64* host_coeff);
void decrypt_coeff(Context* c, const Ct& ct, u64* dev_out);  // [l][N] coefficient domain

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
