// capi.cu -- the extern "C" boundary (include/gwhe.h).  Marshals arguments,
// converts exceptions into status codes and keeps the last error text.
#include <algorithm>
#include <cstring>

#include "capi_types.cuh"

using namespace gwhe;

namespace {

// Runs f with exceptions turned into status codes.  A call on a context is
// refused (GWHE_EINVAL) unless the context's device is current: its tables,
// keys and pool live there.
template <class F>
int guard(Context* c, F&& f) {
  try {
    if (c) require_device(c);
    f();
    return GWHE_OK;
  } catch (const Error& e) {
    if (c) c->last_error = e.what();
    return e.code;
  } catch (const std::exception& e) {
    if (c) c->last_error = e.what();
    return GWHE_EINVAL;
  }
}

Context* C(gwhe_ctx* x) { return x ? x->c : nullptr; }

void need(bool cond, const char* msg) {
  if (!cond) throw Error(ST_EINVAL, msg);
}

void sync(Context* c) { GWHE_CUDA(cudaStreamSynchronize(c->stream)); }

}  // namespace

extern "C" {

int gwhe_gen_primes(const gwhe_params* prm, uint64_t* q, uint64_t* p) {
  if (!prm || !q || !p) return GWHE_EINVAL;
  return gen_primes(prm->logN, prm->L, prm->q0_bits, prm->scale_bits, prm->K, prm->sp_bits, q, p);
}

int gwhe_fft_twiddles(int logN, int sign, double* W, double* T) {
  if (logN < 2 || logN > 17 || !W || !T || (sign != 1 && sign != -1)) return GWHE_EINVAL;
  fft_twiddles(logN, sign, W, T);
  return GWHE_OK;
}

int gwhe_layout(int logN, int n, long k, long out[5]) {
  return guard(nullptr, [&] {
    need(out && logN >= 2 && logN <= 20, "bad arguments");
    Layout L = make_layout(logN, n, 1, k);
    out[0] = L.nb;
    out[1] = L.B;
    out[2] = L.tau;
    out[3] = L.batches;
    out[4] = L.H;
  });
}

int gwhe_ctx_create(const gwhe_params* prm, uint64_t seed, void* stream, gwhe_ctx** out) {
  if (!out || !prm) return GWHE_EINVAL;
  *out = nullptr;
  Context* c = nullptr;
  std::string err;
  int rc = GWHE_OK;
  try {
    Params P{prm->logN, prm->L, prm->q0_bits, prm->scale_bits, prm->K, prm->sp_bits, prm->dnum};
    c = ctx_create(P, seed, (cudaStream_t)stream);
  } catch (const Error& e) {
    rc = e.code;
  } catch (const std::exception&) {
    rc = GWHE_EINVAL;
  }
  if (rc != GWHE_OK) return rc;
  *out = new gwhe_ctx{c};
  return GWHE_OK;
}

int gwhe_ctx_destroy(gwhe_ctx* ctx) {
  if (!ctx) return GWHE_EINVAL;
  ctx_destroy(ctx->c);
  delete ctx;
  return GWHE_OK;
}

const char* gwhe_last_error(const gwhe_ctx* ctx) {
  return (ctx && ctx->c) ? ctx->c->last_error.c_str() : "no context";
}

int gwhe_ctx_moduli(const gwhe_ctx* ctx, uint64_t* out) {
  if (!ctx || !out) return GWHE_EINVAL;
  std::memcpy(out, ctx->c->mod.data(), sizeof(uint64_t) * ctx->c->mod.size());
  return GWHE_OK;
}

int gwhe_ctx_set_stream(gwhe_ctx* ctx, void* stream) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    const cudaStream_t ns = (cudaStream_t)stream;
    if (ns == c->stream) return;
    // work queued so far on the old stream comes first on the new one
    cudaEvent_t e;
    GWHE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t r = cudaEventRecord(e, c->stream);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(ns, e, 0);
    cudaEventDestroy(e);
    GWHE_CUDA(r);
    c->stream = ns;
  });
}

int gwhe_sync(gwhe_ctx* ctx) {
  return guard(C(ctx), [&] { sync(C(ctx)); });
}

int gwhe_keygen(gwhe_ctx* ctx, const int32_t* rot_steps, size_t nrot, int conj) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    std::vector<u32> gal;
    for (size_t i = 0; i < nrot; ++i) {
      const u32 g = galois_for_rotation(c, rot_steps[i]);
      if (std::find(gal.begin(), gal.end(), g) == gal.end() && g != 1) gal.push_back(g);
    }
    if (conj) gal.push_back(galois_conj(c));
    keygen(c, gal);
    sync(c);
  });
}

// npoly polynomials of nl NTT-domain rows (row i modulo mod[pidx[i]], or
// mod[first_mod + i] without pidx) -> coefficient domain, host
static void export_rows(Context* c, const u64* dev, int npoly, int nl, int first_mod, u64* host,
                        const int* pidx = nullptr) {
  const size_t N = c->N, words = (size_t)npoly * nl * N;
  Tmp t(c, sizeof(u64) * words);
  GWHE_CUDA(cudaMemcpyAsync(t.p, dev, sizeof(u64) * words, cudaMemcpyDeviceToDevice, c->stream));
  RowMap rm;
  rm.npoly = npoly;
  rm.nl = nl;
  rm.poly_stride = nl;
  for (int i = 0; i < nl; ++i) {
    rm.off[i] = (uint16_t)i;
    rm.pidx[i] = (uint8_t)(pidx ? pidx[i] : first_mod + i);
  }
  ntt_inverse(c, t.u(), rm);
  GWHE_CUDA(cudaMemcpyAsync(host, t.p, sizeof(u64) * words, cudaMemcpyDeviceToHost, c->stream));
  sync(c);
}

int gwhe_export_secret(gwhe_ctx* ctx, int64_t* s) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(c->d_sk && s, "no secret key");
    std::vector<u64> r(c->N);
    export_rows(c, c->d_sk, 1, 1, 0, r.data());
    const u64 q = c->mod[0];
    for (int k = 0; k < c->N; ++k) s[k] = r[k] > q / 2 ? -(int64_t)(q - r[k]) : (int64_t)r[k];
  });
}

int gwhe_export_pk(gwhe_ctx* ctx, uint64_t* pk) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(c->d_pk && pk, "no public key");
    export_rows(c, c->d_pk, 2, c->P.L, 0, pk);
  });
}

int gwhe_export_ksk(gwhe_ctx* ctx, uint32_t key_id, int k, uint64_t* out) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    auto it = c->ksk.find(key_id);
    if (it == c->ksk.end()) throw Error(ST_ENOKEY, "no such key");
    need(k >= 1 && k <= kMaxSpecial && it->second.fam[k].d, "no key family with that count");
    const Ksk& f = it->second.fam[k];
    std::vector<int> pidx(f.rows());
    for (int u = 0; u < f.rows(); ++u) pidx[u] = u < f.lmax ? u : c->P.L + (u - f.lmax);
    export_rows(c, f.d, 2 * f.dk, f.rows(), 0, out, pidx.data());
  });
}

int gwhe_ks_special(const gwhe_ctx* ctx, int l, int* k, int* key_lmax) {
  if (!ctx || !ctx->c || !k) return GWHE_EINVAL;
  const Context* c = ctx->c;
  if (l < 1 || l > c->P.L) return GWHE_EINVAL;
  *k = c->ks_k[l];
  if (key_lmax) *key_lmax = c->key_lmax[*k];
  return GWHE_OK;
}

int gwhe_ct_create(gwhe_ctx* ctx, int npoly, int cap, gwhe_ct** out) {
  if (!out) return GWHE_EINVAL;
  *out = nullptr;
  return guard(C(ctx), [&] {
    need(npoly == 2 || npoly == 3, "npoly must be 2 or 3");
    need(cap >= 1 && cap <= C(ctx)->P.L, "cap must be in [1, L]");
    std::unique_ptr<gwhe_ct> h(new gwhe_ct{ctx, ct_new(C(ctx), npoly, cap, cap, 1.0)});
    *out = h.release();
  });
}

int gwhe_ct_destroy(gwhe_ct* ct) {
  if (!ct) return GWHE_EINVAL;
  delete ct;
  return GWHE_OK;
}

int gwhe_ct_info(const gwhe_ct* ct, int* npoly, int* l, double* scale) {
  if (!ct) return GWHE_EINVAL;
  if (npoly) *npoly = ct->ct->npoly;
  if (l) *l = ct->ct->l;
  if (scale) *scale = ct->ct->scale;
  return GWHE_OK;
}

int gwhe_ct_import(gwhe_ct* ct, const uint64_t* coeffs, int npoly, int l, double scale) {
  if (!ct) return GWHE_EINVAL;
  return guard(C(ct->owner), [&] {
    need(coeffs && l >= 1, "bad import");
    ct_import(C(ct->owner), *ct->ct, coeffs, npoly, l, scale);
  });
}

int gwhe_ct_export(const gwhe_ct* ct, uint64_t* coeffs) {
  if (!ct) return GWHE_EINVAL;
  return guard(C(ct->owner), [&] {
    need(coeffs, "null output");
    ct_export(C(ct->owner), *ct->ct, coeffs);
  });
}

int gwhe_encode(gwhe_ctx* ctx, const double* z, double scale, int64_t* coeffs) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    const int M = c->N / 2;
    Tmp dz(c, sizeof(double2) * M), work(c, sizeof(double2) * M), out(c, sizeof(i64) * c->N);
    GWHE_CUDA(cudaMemcpyAsync(dz.p, z, sizeof(double2) * M, cudaMemcpyHostToDevice, c->stream));
    encode_batch(c, dz.as<double2>(), 1, scale, out.as<i64>(), work.as<double2>());
    GWHE_CUDA(cudaMemcpyAsync(coeffs, out.p, sizeof(i64) * c->N, cudaMemcpyDeviceToHost, c->stream));
    sync(c);
  });
}

int gwhe_encode_batch(gwhe_ctx* ctx, const double* z_dev, int count, double scale,
                      int64_t* coeffs_dev) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(z_dev && coeffs_dev && count >= 1, "bad arguments");
    Tmp work(c, sizeof(double2) * (size_t)count * (c->N / 2));
    encode_batch(c, (const double2*)z_dev, count, scale, coeffs_dev, work.as<double2>());
  });
}

int gwhe_encrypt(gwhe_ctx* ctx, const double* z, double scale, int l, uint64_t enc_id, gwhe_ct* out) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(out && out->ct->npoly == 2 && l >= 1 && l <= out->ct->cap, "bad output ciphertext");
    const int M = c->N / 2;
    Tmp dz(c, sizeof(double2) * M);
    GWHE_CUDA(cudaMemcpyAsync(dz.p, z, sizeof(double2) * M, cudaMemcpyHostToDevice, c->stream));
    encrypt_slots(c, dz.as<double2>(), 1, scale, l, enc_id, out->ct->d, out->ct->cap);
    out->ct->l = l;
    out->ct->scale = scale;
    sync(c);
  });
}

int gwhe_encrypt_coeffs(gwhe_ctx* ctx, const int64_t* m, double scale, int l, uint64_t enc_id,
                        gwhe_ct* out) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(out && out->ct->npoly == 2 && l >= 1 && l <= out->ct->cap, "bad output ciphertext");
    Tmp dm(c, sizeof(i64) * c->N);
    GWHE_CUDA(cudaMemcpyAsync(dm.p, m, sizeof(i64) * c->N, cudaMemcpyHostToDevice, c->stream));
    encrypt_coeffs(c, dm.as<i64>(), 1, l, enc_id, out->ct->d, out->ct->cap);
    out->ct->l = l;
    out->ct->scale = scale;
    sync(c);
  });
}

int gwhe_decrypt(gwhe_ctx* ctx, const gwhe_ct* ct, uint64_t* m) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(ct && m && ct->ct->npoly == 2, "bad ciphertext");
    Tmp t(c, sizeof(u64) * ct->ct->l * c->N);
    decrypt_coeff(c, *ct->ct, t.u());
    GWHE_CUDA(cudaMemcpyAsync(m, t.p, sizeof(u64) * ct->ct->l * c->N, cudaMemcpyDeviceToHost,
                              c->stream));
    sync(c);
  });
}

int gwhe_decrypt_decode(gwhe_ctx* ctx, const gwhe_ct* ct, double* z) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(ct && z && ct->ct->npoly == 2, "bad ciphertext");
    const int M = c->N / 2;
    Ct v = *ct->ct;
    v.owned = false;
    v.l = 1;
    Tmp m(c, sizeof(u64) * c->N), out(c, sizeof(double2) * M), work(c, sizeof(double2) * M);
    decrypt_coeff(c, v, m.u());
    decode_batch(c, m.u(), 1, ct->ct->scale, out.as<double2>(), work.as<double2>());
    GWHE_CUDA(cudaMemcpyAsync(z, out.p, sizeof(double2) * M, cudaMemcpyDeviceToHost, c->stream));
    sync(c);
  });
}

#define CT(x) (*(x)->ct)

int gwhe_add(gwhe_ctx* ctx, const gwhe_ct* a, const gwhe_ct* b, gwhe_ct* out) {
  return guard(C(ctx), [&] { op_addsub(C(ctx), CT(a), CT(b), CT(out), false); });
}
int gwhe_sub(gwhe_ctx* ctx, const gwhe_ct* a, const gwhe_ct* b, gwhe_ct* out) {
  return guard(C(ctx), [&] { op_addsub(C(ctx), CT(a), CT(b), CT(out), true); });
}
int gwhe_negate(gwhe_ctx* ctx, const gwhe_ct* a, gwhe_ct* out) {
  return guard(C(ctx), [&] { op_negate(C(ctx), CT(a), CT(out)); });
}
int gwhe_add_const(gwhe_ctx* ctx, gwhe_ct* ct, double v) {
  return guard(C(ctx), [&] { op_add_const(C(ctx), CT(ct), v); });
}
int gwhe_mul_int(gwhe_ctx* ctx, gwhe_ct* ct, int64_t k) {
  return guard(C(ctx), [&] { op_mul_int(C(ctx), CT(ct), k); });
}
int gwhe_mul_const(gwhe_ctx* ctx, gwhe_ct* ct, double v) {
  return guard(C(ctx), [&] { op_mul_const(C(ctx), CT(ct), v); });
}
int gwhe_mul_mask(gwhe_ctx* ctx, const gwhe_ct* a, const double* z, gwhe_ct* out) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    const int M = c->N / 2, l = CT(a).l;
    need(l >= 2, "no level left for a mask product");
    const double ql = (double)c->mod[l - 1];
    Tmp dz(c, sizeof(double2) * M), pt(c, sizeof(u64) * l * c->N);
    GWHE_CUDA(cudaMemcpyAsync(dz.p, z, sizeof(double2) * M, cudaMemcpyHostToDevice, c->stream));
    encode_to_ntt(c, dz.as<double2>(), 1, ql, l, pt.u());
    op_mul_plain(c, CT(a), pt.u(), ql, CT(out));
    op_rescale(c, CT(out));
    sync(c);
  });
}
int gwhe_tensor(gwhe_ctx* ctx, const gwhe_ct* a, const gwhe_ct* b, gwhe_ct* out) {
  return guard(C(ctx), [&] { op_tensor_mac(C(ctx), {{a->ct.get(), b->ct.get()}}, CT(out)); });
}
int gwhe_tensor_sum(gwhe_ctx* ctx, const gwhe_ct* const* a, const gwhe_ct* const* b, size_t n,
                    gwhe_ct* out) {
  return guard(C(ctx), [&] {
    need(n > 0, "empty sum");
    std::vector<std::pair<const Ct*, const Ct*>> terms;
    for (size_t i = 0; i < n; ++i) terms.push_back({a[i]->ct.get(), b[i]->ct.get()});
    op_tensor_mac(C(ctx), terms, CT(out));
  });
}
int gwhe_relin(gwhe_ctx* ctx, const gwhe_ct* t3, gwhe_ct* out) {
  return guard(C(ctx), [&] { op_relin(C(ctx), CT(t3), CT(out)); });
}
int gwhe_rescale(gwhe_ctx* ctx, gwhe_ct* ct) {
  return guard(C(ctx), [&] { op_rescale(C(ctx), CT(ct)); });
}
int gwhe_mult(gwhe_ctx* ctx, const gwhe_ct* a, const gwhe_ct* b, gwhe_ct* out) {
  return guard(C(ctx), [&] { op_mult(C(ctx), CT(a), CT(b), CT(out)); });
}
int gwhe_rotate(gwhe_ctx* ctx, const gwhe_ct* a, int steps, gwhe_ct* out) {
  return guard(C(ctx), [&] { op_rotate(C(ctx), CT(a), steps, CT(out)); });
}
int gwhe_rotate_sum(gwhe_ctx* ctx, const gwhe_ct* a, const int32_t* steps, int nsteps,
                    gwhe_ct* out) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(a && out && steps && nsteps >= 1 && nsteps <= kMaxHoist, "bad rotation sum");
    const Ct& x = *a->ct;
    need(x.npoly == 2 && out->ct->npoly == 2 && out->ct->cap >= x.l, "bad ciphertexts");
    CtSetPtr s = set_new(c, 1, 2, x.l, x.l, x.scale);
    for (int p = 0; p < 2; ++p)
      GWHE_CUDA(cudaMemcpyAsync(s->item(0) + (size_t)p * x.l * c->N, x.poly(p),
                                sizeof(u64) * x.l * c->N, cudaMemcpyDeviceToDevice, c->stream));
    set_rotate_sum(c, *s, std::vector<int>(steps, steps + nsteps));
    Ct& o = *out->ct;
    for (int p = 0; p < 2; ++p)
      GWHE_CUDA(cudaMemcpyAsync(o.poly(p), s->item(0) + (size_t)p * x.l * c->N,
                                sizeof(u64) * x.l * c->N, cudaMemcpyDeviceToDevice, c->stream));
    o.l = x.l;
    o.scale = x.scale;
  });
}

int gwhe_rotate_sum_batch(gwhe_ctx* ctx, const gwhe_ct* const* a, int count,
                          const int32_t* steps, int nsteps, gwhe_ct* const* out) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(a && out && steps && count >= 1 && nsteps >= 1 && nsteps <= kMaxHoist,
         "bad rotation sum batch");
    const Ct& x0 = *a[0]->ct;
    for (int i = 0; i < count; ++i) {
      const Ct& x = *a[i]->ct;
      need(x.npoly == 2 && x.l == x0.l && x.scale == x0.scale, "inputs must share level and scale");
      need(out[i]->ct->npoly == 2 && out[i]->ct->cap >= x.l, "output too small");
    }
    const size_t N = c->N;
    const int l = x0.l;
    CtSetPtr s = set_new(c, count, 2, l, l, x0.scale);
    for (int i = 0; i < count; ++i)
      for (int p = 0; p < 2; ++p)
        GWHE_CUDA(cudaMemcpyAsync(s->item(i) + (size_t)p * l * N, a[i]->ct->poly(p),
                                  sizeof(u64) * l * N, cudaMemcpyDeviceToDevice, c->stream));
    set_rotate_sum(c, *s, std::vector<int>(steps, steps + nsteps));
    for (int i = 0; i < count; ++i) {
      Ct& o = *out[i]->ct;
      for (int p = 0; p < 2; ++p)
        GWHE_CUDA(cudaMemcpyAsync(o.poly(p), s->item(i) + (size_t)p * l * N, sizeof(u64) * l * N,
                                  cudaMemcpyDeviceToDevice, c->stream));
      o.l = l;
      o.scale = x0.scale;
    }
  });
}

int gwhe_rotate_batch(gwhe_ctx* ctx, const gwhe_ct* const* a, int count, int32_t step,
                      int rescale, gwhe_ct* const* out) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(a && out && count >= 1, "bad rotation batch");
    const Ct& x0 = *a[0]->ct;
    const int l = x0.l;
    need(!rescale || l >= 2, "no level left to rescale");
    for (int i = 0; i < count; ++i) {
      const Ct& x = *a[i]->ct;
      need(x.npoly == 2 && x.l == l && x.scale == x0.scale, "inputs must share level and scale");
      need(out[i]->ct->npoly == 2 && out[i]->ct->cap >= l, "output too small");
    }
    const size_t N = c->N;
    CtSetPtr s = set_new(c, count, 2, l, l, x0.scale);
    for (int i = 0; i < count; ++i)
      for (int p = 0; p < 2; ++p)
        GWHE_CUDA(cudaMemcpyAsync(s->item(i) + (size_t)p * l * N, a[i]->ct->poly(p),
                                  sizeof(u64) * l * N, cudaMemcpyDeviceToDevice, c->stream));
    CtSetPtr r = set_new(c, count, 2, l, l, x0.scale);
    set_galois(c, *s, galois_for_rotation(c, step), *r);
    if (rescale) set_rescale(c, *r);
    for (int i = 0; i < count; ++i) {
      Ct& o = *out[i]->ct;
      for (int p = 0; p < 2; ++p)
        GWHE_CUDA(cudaMemcpyAsync(o.poly(p), r->item(i) + (size_t)p * r->cap * N,
                                  sizeof(u64) * r->l * N, cudaMemcpyDeviceToDevice, c->stream));
      o.l = r->l;
      o.scale = r->scale;
    }
  });
}

int gwhe_conjugate(gwhe_ctx* ctx, const gwhe_ct* a, gwhe_ct* out) {
  return guard(C(ctx), [&] { op_conj(C(ctx), CT(a), CT(out)); });
}
int gwhe_drop(gwhe_ct* ct, int l) {
  if (!ct) return GWHE_EINVAL;
  return guard(C(ct->owner), [&] { op_drop(CT(ct), l); });
}

int gwhe_keyswitch(gwhe_ctx* ctx, const uint64_t* x, int l, uint32_t key_id, uint64_t* out) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(x && out && l >= 1 && l <= c->P.L, "bad arguments");
    auto it = c->ksk.find(key_id);
    if (it == c->ksk.end()) throw Error(ST_ENOKEY, "no such key");
    const size_t N = c->N;
    Tmp dx(c, sizeof(u64) * l * N), dout(c, sizeof(u64) * 2 * l * N);
    GWHE_CUDA(cudaMemcpyAsync(dx.p, x, sizeof(u64) * l * N, cudaMemcpyHostToDevice, c->stream));
    ntt_forward(c, dx.u(), rows_q(1, l, l));
    keyswitch(c, dx.u(), l, it->second, dout.u(), dout.u() + (size_t)l * N, nullptr, nullptr);
    ntt_inverse(c, dout.u(), rows_q(2, l, l));
    GWHE_CUDA(cudaMemcpyAsync(out, dout.p, sizeof(u64) * 2 * l * N, cudaMemcpyDeviceToHost,
                              c->stream));
    sync(c);
  });
}

int gwhe_ntt_batch(gwhe_ctx* ctx, uint64_t* dev, int npoly, int nlimbs, int inverse) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(dev && npoly >= 1 && nlimbs >= 1 && nlimbs <= c->nmod && nlimbs <= kMaxRowLimbs,
         "bad arguments");
    RowMap rm = rows_q(npoly, nlimbs, nlimbs);
    if (inverse)
      ntt_inverse(c, dev, rm);
    else
      ntt_forward(c, dev, rm);
  });
}

int gwhe_job_create_ex(gwhe_ctx* ctx, int n, int d, long k, int layout, gwhe_job** out) {
  if (!out) return GWHE_EINVAL;
  *out = nullptr;
  return guard(C(ctx), [&] {
    std::unique_ptr<gwhe_job> j(new gwhe_job());
    j->owner = ctx;
    j->job.reset(job_create(C(ctx), n, d, k, layout));
    *out = j.release();
  });
}

int gwhe_job_create(gwhe_ctx* ctx, int n, int d, long k, gwhe_job** out) {
  return gwhe_job_create_ex(ctx, n, d, k, GWHE_LAYOUT_AUTO, out);
}

int gwhe_job_info(const gwhe_job* job, long out[8]) {
  if (!job || !out || !job->job) return GWHE_EINVAL;
  const Job* j = job->job.get();
  const Layout& L = j->lay;
  const long v[8] = {L.M, L.nb, L.B, L.tau, j->factored ? 0 : L.H, L.batches,
                     j->factored ? GWHE_LAYOUT_FACTORED : GWHE_LAYOUT_MCCP,
                     j->factored ? kFactLevel : kBatchLevel};
  for (int i = 0; i < 8; ++i) out[i] = v[i];
  return GWHE_OK;
}

int gwhe_job_rotation_steps(const gwhe_job* job, int32_t* steps, int cap, int* count) {
  if (!job || !count || !job->job) return GWHE_EINVAL;
  const std::vector<int> s = job_rotation_steps(job->job.get());
  *count = (int)s.size();
  if (steps) {
    if (cap < (int)s.size()) return GWHE_EINVAL;
    for (size_t i = 0; i < s.size(); ++i) steps[i] = s[i];
  }
  return GWHE_OK;
}

int gwhe_job_destroy(gwhe_job* job) {
  if (!job) return GWHE_EINVAL;
  Context* c = C(job->owner);
  delete job;
  if (c) cudaStreamSynchronize(c->stream);
  return GWHE_OK;
}

int gwhe_encrypt_inputs(gwhe_job* job, const double* X, const double* XtX_inv, const double* y) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] {
    need(X && XtX_inv && y, "null input");
    job_encrypt_inputs(job->job.get(), X, XtX_inv, y);
  });
}

int gwhe_encrypt_covariates(gwhe_job* job, const double* X, const double* XtX_inv) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] {
    need(X && XtX_inv, "null input");
    job_encrypt_covariates(job->job.get(), X, XtX_inv);
  });
}

int gwhe_encrypt_phenotype(gwhe_job* job, const double* y) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] {
    need(y != nullptr, "null input");
    job_encrypt_phenotype(job->job.get(), y);
  });
}

int gwhe_encrypt_snps(gwhe_job* job, const double* S, long b0, long b1) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] {
    need(S != nullptr, "null input");
    job_encrypt_snps(job->job.get(), S, b0, b1);
  });
}

int gwhe_fit_covariates(gwhe_job* job, int kappa) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] { job_fit(job->job.get(), kappa); });
}

int gwhe_set_fit_state(gwhe_job* job, const double* M, const double* w, const double* wz) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] {
    need(M && w && wz, "null input");
    job_set_fit_state(job->job.get(), M, w, wz);
  });
}

int gwhe_snp_stats(gwhe_job* job, const double* S, long b0, long b1, int keep) {
  (void)keep;
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] { job_snp_stats(job->job.get(), S, b0, b1); });
}

int gwhe_decrypt_results(gwhe_job* job, double* num, double* den) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] {
    need(num && den, "null output");
    job_decrypt(job->job.get(), num, den);
  });
}

int gwhe_job_ct(gwhe_job* job, int which, long index, gwhe_ct** view) {
  if (!job || !view) return GWHE_EINVAL;
  *view = nullptr;
  return guard(C(job->owner), [&] {
    Job* j = job->job.get();
    const Ct* src = nullptr;
    switch (which) {
      case 0:
      case 1:
      case 2:
        need(index >= 0 && index < (long)j->out.size() && j->out[index][which], "no such batch");
        src = j->out[index][which].get();
        break;
      case 3:
        need(index >= 0 && index < (long)j->DupM.size(), "no such column");
        src = j->DupM[index].get();
        break;
      case 4: src = j->DupW.get(); break;
      case 5: src = j->DupWZ.get(); break;
      case 6: src = j->zp.get(); break;
      case 7: src = j->beta.get(); break;
      case 8:
        need(index >= 0 && index < (long)j->Mct.size(), "no such M ciphertext");
        src = j->Mct[index].get();
        break;
      case 9: src = j->z.get(); break;
      case 10: src = j->w_m.get(); break;
      case 11:
        need(index >= 0 && index < (long)j->DupX.size(), "no such Dup(X_c)");
        src = j->DupX[index].get();
        break;
      case 12:
        need(index >= 0 && index < (long)j->DupB.size(), "no such Dup((XA)_c)");
        src = j->DupB[index].get();
        break;
      default: break;
    }
    need(src != nullptr, "no such ciphertext");
    CtPtr v(new Ct(*src));
    v->owned = false;
    *view = new gwhe_ct{job->owner, std::move(v)};
  });
}

int gwhe_job_state_size(const gwhe_job* job, size_t* words) {
  if (!job || !words) return GWHE_EINVAL;
  return guard(C(job->owner), [&] { *words = job_state_words(job->job.get()); });
}

int gwhe_job_export_state(const gwhe_job* job, uint64_t* buf, size_t words) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] {
    need(buf != nullptr, "null buffer");
    job_export_state(job->job.get(), buf, words);
  });
}

int gwhe_job_import_state(gwhe_job* job, const uint64_t* buf, size_t words) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] {
    need(buf != nullptr, "null buffer");
    job_import_state(job->job.get(), buf, words);
  });
}

int gwhe_job_set_nonce(gwhe_job* job, uint32_t nonce) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] { job_set_nonce(job->job.get(), nonce); });
}

int gwhe_job_set_host_state(gwhe_job* job, int chunk) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] { job_set_host_state(job->job.get(), chunk); });
}

int gwhe_job_release_results(gwhe_job* job) {
  if (!job) return GWHE_EINVAL;
  return guard(C(job->owner), [&] { job_release_results(job->job.get()); });
}

int gwhe_ctx_create_child(gwhe_ctx* ctx, void* stream, gwhe_ctx** out) {
  if (!out) return GWHE_EINVAL;
  *out = nullptr;
  return guard(C(ctx), [&] {
    std::unique_ptr<gwhe_ctx> h(new gwhe_ctx());
    h->c = ctx_child(C(ctx), (cudaStream_t)stream);
    *out = h.release();
  });
}

int gwhe_set_ntt_variant(gwhe_ctx* ctx, int variant) {
  return guard(C(ctx), [&] {
    need(variant >= 0 && variant < kNttVariants, "no such transform shape");
    C(ctx)->ntt_variant = variant;
    C(ctx)->ntt_variant_small = variant;
  });
}

int gwhe_autotune(gwhe_ctx* ctx, int rows, double* ms, int* chosen) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    need(rows >= 1 && rows <= 4096, "rows must be in [1, 4096]");
    for (int v = 0; v < kNttVariants; ++v)
      if (ms) ms[v] = 0.0;
    if (c->logN != 16) {  // one shape only
      if (chosen) *chosen = rows >= kNttSmallRows ? c->ntt_variant : c->ntt_variant_small;
      return;
    }
    // zero residues are valid inputs; the transforms' cost does not depend on
    // the values
    Tmp buf(c, sizeof(u64) * (size_t)rows * c->N);
    GWHE_CUDA(cudaMemsetAsync(buf.p, 0, sizeof(u64) * (size_t)rows * c->N, c->stream));
    RowMap rm;
    rm.npoly = rows;
    rm.nl = 1;
    rm.poly_stride = 1;
    rm.off[0] = 0;
    rm.pidx[0] = 0;
    cudaEvent_t e0, e1;
    GWHE_CUDA(cudaEventCreate(&e0));
    GWHE_CUDA(cudaEventCreate(&e1));
    int best = 0;
    double best_ms = 1e30;
    // the size class being tuned: launches of at least kNttSmallRows rows,
    // or the smaller ones
    int& slot = rows >= kNttSmallRows ? c->ntt_variant : c->ntt_variant_small;
    for (int v = 0; v < kNttVariants; ++v) {
      slot = v;
      ntt_forward(c, buf.u(), rm);
      ntt_inverse(c, buf.u(), rm);
      float t = 1e30f;
      for (int rep = 0; rep < (rows < kNttSmallRows ? 10 : 3); ++rep) {
        GWHE_CUDA(cudaEventRecord(e0, c->stream));
        ntt_forward(c, buf.u(), rm);
        ntt_inverse(c, buf.u(), rm);
        GWHE_CUDA(cudaEventRecord(e1, c->stream));
        GWHE_CUDA(cudaEventSynchronize(e1));
        float x = 0.f;
        GWHE_CUDA(cudaEventElapsedTime(&x, e0, e1));
        t = std::min(t, x);
      }
      if (ms) ms[v] = t;
      if (t < best_ms) {
        best_ms = t;
        best = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    slot = best;
    if (chosen) *chosen = best;
  });
}

int gwhe_ks_histogram(const gwhe_ctx* ctx, long* out, int n) {
  if (!ctx || !out || n < 1) return GWHE_EINVAL;
  for (int l = 0; l < n; ++l) out[l] = l <= kMaxRowLimbs ? ctx->c->ks_by_level[l] : 0;
  return GWHE_OK;
}

long gwhe_launch_count(const gwhe_ctx* ctx) { return (ctx && ctx->c) ? ctx->c->launches : -1; }

int gwhe_prof_enable(gwhe_ctx* ctx, int on) {
  return guard(C(ctx), [&] {
    Context* c = C(ctx);
    double ms[PROF_NCAT], by[PROF_NCAT];
    long n[PROF_NCAT];
    prof_read(c, ms, by, n);  // discard what was recorded so far
    c->prof.on = on != 0;
  });
}

int gwhe_prof_read(gwhe_ctx* ctx, double* ms, double* bytes, long* count) {
  return guard(C(ctx), [&] {
    need(ms && bytes && count, "null output");
    prof_read(C(ctx), ms, bytes, count);
  });
}

int gwhe_device_ok(int context_device, int current_device) {
  return device_check(context_device, current_device);
}

int gwhe_ctx_device(const gwhe_ctx* ctx, int* device) {
  if (!ctx || !ctx->c || !device) return GWHE_EINVAL;
  *device = ctx->c->device;
  return GWHE_OK;
}

int gwhe_mem_info(gwhe_ctx* ctx, uint64_t out[4]) {
  return guard(C(ctx), [&] {
    need(out != nullptr, "null output");
    cudaMemPool_t pool;
    GWHE_CUDA(cudaDeviceGetDefaultMemPool(&pool, C(ctx)->device));
    uint64_t used = 0, reserved = 0;
    GWHE_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    GWHE_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
    size_t fr = 0, tot = 0;
    GWHE_CUDA(cudaMemGetInfo(&fr, &tot));
    out[0] = used;
    out[1] = reserved;
    out[2] = fr;
    out[3] = tot;
  });
}

long gwhe_job_keyswitches(const gwhe_job* job) {
  return (job && job->owner) ? job->owner->c->ks_count : -1;
}

}  // extern "C"
