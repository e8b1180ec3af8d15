// ckks.cu -- RNS-CKKS context, key generation and evaluator (host
// orchestration of the kernels in ntt.cu / kernels.cu).
//
// Conventions shared with the documented spec of the library header:
//   scale of a product = product of scales; rescale divides by (double)q_last;
//   a sum keeps the first operand's scale (relative mismatch above 2^-10 is an
//   error); a real constant c multiplies as round(c * q_last) then rescales.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ckks.cuh"

namespace gwhe {

// ---------------------------------------------------------------- memory
void* dalloc_bytes(Context* c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMallocAsync(&p, bytes, c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(ST_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  return p;
}
u64* dalloc_u64(Context* c, size_t words) { return (u64*)dalloc_bytes(c, words * sizeof(u64)); }
void dfree(Context* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}

ProfScope::ProfScope(Context* c_, int cat_, double bytes_) : c(c_), cat(cat_), bytes(bytes_) {
  if (!c->prof.on) return;
  if (c->prof.pool.empty()) {
    cudaEvent_t e;
    GWHE_CUDA(cudaEventCreate(&e));
    c->prof.pool.push_back(e);
  }
  a = c->prof.pool.back();
  c->prof.pool.pop_back();
  cudaEventRecord(a, c->stream);
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b;
  if (c->prof.pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) return;
  } else {
    b = c->prof.pool.back();
    c->prof.pool.pop_back();
  }
  cudaEventRecord(b, c->stream);
  c->prof.recs.push_back(ProfRec{a, b, bytes, cat});
}

void prof_read(Context* c, double* ms, double* bytes, long* count) {
  for (int i = 0; i < PROF_NCAT; ++i) {
    ms[i] = 0;
    bytes[i] = 0;
    count[i] = 0;
  }
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
  for (const ProfRec& r : c->prof.recs) {
    float t = 0;
    GWHE_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.cat] += t;
    bytes[r.cat] += r.bytes;
    count[r.cat] += 1;
    c->prof.pool.push_back(r.a);
    c->prof.pool.push_back(r.b);
  }
  c->prof.recs.clear();
}

Tmp::Tmp(Context* c_, size_t bytes) : c(c_), p(dalloc_bytes(c_, bytes)) {}
Tmp::~Tmp() { dfree(c, p); }

Ct::~Ct() {
  if (owned && d && ctx) dfree(ctx, d);
}
u64* Ct::poly(int p) const { return d + (size_t)p * cap * ctx->N; }
u64* Ct::limb(int p, int i) const { return d + ((size_t)p * cap + i) * ctx->N; }

static PolyView pv(const Ct& a) { return PolyView{a.d, a.cap}; }
static CPolyView cpv(const Ct& a) { return CPolyView{a.d, a.cap}; }

CtPtr ct_new(Context* c, int npoly, int cap, int l, double scale) {
  CtPtr ct(new Ct());
  ct->ctx = c;
  ct->npoly = npoly;
  ct->cap = cap;
  ct->l = l;
  ct->scale = scale;
  ct->d = dalloc_u64(c, (size_t)npoly * cap * c->N);
  return ct;
}

CtPtr ct_clone(Context* c, const Ct& a) {
  CtPtr ct = ct_new(c, a.npoly, a.l, a.l, a.scale);
  for (int p = 0; p < a.npoly; ++p)
    GWHE_CUDA(cudaMemcpyAsync(ct->poly(p), a.poly(p), sizeof(u64) * a.l * c->N,
                              cudaMemcpyDeviceToDevice, c->stream));
  return ct;
}

// ---------------------------------------------------------------- context
template <class T>
static T* upload(Context* c, const std::vector<T>& v) {
  T* d = nullptr;
  GWHE_CUDA(cudaMalloc(&d, sizeof(T) * std::max<size_t>(v.size(), 1)));
  GWHE_CUDA(cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return d;
}

Context* ctx_create(const Params& P, u64 seed, cudaStream_t stream) {
  GWHE_REQUIRE(P.logN >= 4 && P.logN <= 17, ST_EINVAL, "logN must be in [4, 17]");
  GWHE_REQUIRE(P.L >= 1 && P.L <= kMaxRowLimbs && P.K >= 1 && P.K <= 16, ST_EINVAL,
               "need 1 <= L <= 64 and 1 <= K <= 16");
  GWHE_REQUIRE(P.dnum >= 1 && P.dnum <= P.L, ST_EINVAL, "need 1 <= dnum <= L");
  GWHE_REQUIRE(P.dnum <= 4, ST_EINVAL, "at most 4 key-switching digits are supported");
  GWHE_REQUIRE(P.L + P.K <= kMaxMod, ST_EINVAL, "too many moduli");
  GWHE_REQUIRE(P.q0_bits <= 60 && P.sp_bits <= 60 && P.scale_bits <= 60, ST_EINVAL,
               "moduli must stay below 2^60");
  const int alpha = (P.L + P.dnum - 1) / P.dnum;
  GWHE_REQUIRE(alpha <= 16, ST_EINVAL, "digits wider than 16 limbs are not supported");
  // the special modulus P must dominate every digit for the switch noise to stay small
  const int digit_bits = P.q0_bits + (alpha - 1) * (P.scale_bits + 1);
  GWHE_REQUIRE(P.K * P.sp_bits + 4 >= digit_bits, ST_EINVAL,
               "special primes too small for the digit size (need K*sp_bits >= digit bits)");

  std::unique_ptr<Context> c(new Context());
  c->P = P;
  c->logN = P.logN;
  c->N = 1 << P.logN;
  c->alpha = alpha;
  c->nmod = P.L + P.K;
  c->seed = seed;
  c->stream = stream;
  GWHE_CUDA(cudaGetDevice(&c->device));
  // the allocation-free key switch's scratch array: its module is loaded and
  // its memory committed here, on this device, so that the entry point's
  // calls themselves reserve nothing
  c->noalloc_scratch = noalloc_scratch_lookup();
  const int N = c->N, L = P.L, K = P.K, nm = c->nmod;
  c->mod.resize(nm);
  if (gen_primes(P.logN, L, P.q0_bits, P.scale_bits, K, P.sp_bits, c->mod.data(),
                 c->mod.data() + L) != ST_OK)
    throw Error(ST_EINVAL, "prime generation failed");
  for (u64 q : c->mod) c->hmod.push_back(make_devmod(q));
  c->d_mod = upload(c.get(), c->hmod);

  // stream-ordered pool: keep freed blocks for reuse
  cudaMemPool_t pool;
  GWHE_CUDA(cudaDeviceGetDefaultMemPool(&pool, c->device));
  uint64_t thr = UINT64_MAX;
  GWHE_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));

  // N^-1 and ipsi[1] per modulus, for the inverse transforms' scale pairs
  std::vector<u64> h_ninv(nm), h_iw1(nm);
  // NTT tables
  {
    std::vector<ulonglong2> psi((size_t)nm * N), ipsi((size_t)nm * N);
    std::vector<u64> ninv(nm), ninv_sh(nm), pw(N), ipw(N);
    std::vector<ulonglong2> iw1n(nm);
    for (int u = 0; u < nm; ++u) {
      const u64 q = c->mod[u];
      const u64 r = find_psi(q, P.logN), ri = host_inv(r, q);
      pw[0] = ipw[0] = 1;
      for (int k = 1; k < N; ++k) {
        pw[k] = host_mulmod(pw[k - 1], r, q);
        ipw[k] = host_mulmod(ipw[k - 1], ri, q);
      }
      for (int i = 0; i < N; ++i) {
        const int b = bitrev_host(i, P.logN);
        const size_t o = (size_t)u * N + i;
        psi[o] = make_ulonglong2(pw[b], shoup_companion(pw[b], q));
        ipsi[o] = make_ulonglong2(ipw[b], shoup_companion(ipw[b], q));
      }
      ninv[u] = host_inv((u64)N % q, q);
      ninv_sh[u] = shoup_companion(ninv[u], q);
      h_ninv[u] = ninv[u];
      h_iw1[u] = ipsi[(size_t)u * N + 1].x;
      const u64 w1n = host_mulmod(ipsi[(size_t)u * N + 1].x, ninv[u], q);
      iw1n[u] = make_ulonglong2(w1n, shoup_companion(w1n, q));
    }
    c->d_psi = upload(c.get(), psi);
    c->d_ipsi = upload(c.get(), ipsi);
    if (P.logN == 16) {
      // the row pass's last four stages in the transposed order of NttTables
      std::vector<ulonglong2> pb((size_t)nm * kTwBPerMod), ipb((size_t)nm * kTwBPerMod);
      for (int u = 0; u < nm; ++u) {
        size_t off = (size_t)u * kTwBPerMod;
        for (int sp = 4; sp < 8; ++sp) {
          const int nj = 1 << (sp - 4);
          for (int g = 0; g < 256; ++g)
            for (int j = 0; j < nj; ++j)
              for (int r = 0; r < 16; ++r) {
                const size_t src = (size_t)u * N + (1u << (8 + sp)) + ((size_t)g << sp) +
                                   (size_t)r * nj + j;
                const size_t dst = off + ((size_t)g << sp) + 16 * j + r;
                pb[dst] = psi[src];
                ipb[dst] = ipsi[src];
              }
          off += (size_t)256 << sp;
        }
      }
      c->d_psiB = upload(c.get(), pb);
      c->d_ipsiB = upload(c.get(), ipb);
    }
    c->d_ninv = upload(c.get(), ninv);
    c->d_ninv_sh = upload(c.get(), ninv_sh);
    c->d_iw1n = upload(c.get(), iw1n);
  }
  // rescale: entry (l, i) = q_{l-1}^-1 mod q_i for i < l - 1
  {
    std::vector<u64> t((size_t)(L + 1) * L * 2, 0);
    for (int l = 2; l <= L; ++l)
      for (int i = 0; i < l - 1; ++i) {
        const u64 q = c->mod[i];
        const u64 v = host_inv(c->mod[l - 1] % q, q);
        t[((size_t)l * L + i) * 2] = v;
        t[((size_t)l * L + i) * 2 + 1] = shoup_companion(v, q);
      }
    c->d_rescale = upload(c.get(), t);
  }
  // base conversion tables
  // special primes per level (see Context::ks_k): the widest digit's bits
  // (upper bound: sum of bit lengths) plus a 24-bit margin against the
  // special product's bits (lower bound: sum of bit lengths minus one)
  for (int l = 1; l <= L; ++l) {
    int need = 0;
    for (int lo = 0; lo < l; lo += alpha) {
      int bits = 0;
      for (int i = lo; i < std::min(lo + alpha, l); ++i) bits += 64 - __builtin_clzll(c->mod[i]);
      need = std::max(need, bits);
    }
    need += 24;
    int k = K, have = 0;
    for (int kk = 1; kk <= K; ++kk) {
      have += 63 - __builtin_clzll(c->mod[L + kk - 1]);
      if (have >= need) {
        k = kk;
        break;
      }
    }
    c->ks_k[l] = k;
    c->key_lmax[k] = l;
  }
  {
    std::vector<u64> store;
    std::vector<std::pair<ConvTable*, size_t>> fix;
    auto add_table = [&](ConvTable& t, const std::vector<int>& in_mod, const std::vector<int>& out_mod) {
      t.n_in = (int)in_mod.size();
      t.n_out = (int)out_mod.size();
      const size_t base = store.size();
      store.resize(base + 2 * t.n_in + (size_t)t.n_in * t.n_out);
      for (int i = 0; i < t.n_in; ++i) {
        const u64 qi = c->mod[in_mod[i]];
        u64 h = 1;
        for (int i2 = 0; i2 < t.n_in; ++i2)
          if (i2 != i) h = host_mulmod(h, c->mod[in_mod[i2]] % qi, qi);
        const u64 hinv = host_inv(h, qi);
        store[base + i] = hinv;
        store[base + t.n_in + i] = shoup_companion(hinv, qi);
        for (int o = 0; o < t.n_out; ++o) {
          const u64 mo = c->mod[out_mod[o]];
          u64 hm = 1;
          for (int i2 = 0; i2 < t.n_in; ++i2)
            if (i2 != i) hm = host_mulmod(hm, c->mod[in_mod[i2]] % mo, mo);
          store[base + 2 * t.n_in + (size_t)i * t.n_out + o] = hm;
        }
      }
      fix.push_back({&t, base});
    };
    for (int l = 1; l <= L; ++l) {
      const int beta = (l + alpha - 1) / alpha;
      for (int j = 0; j < beta; ++j) {
        const int lo = j * alpha, hi = std::min(lo + alpha, l);
        ConvTable& t = c->modup[{l, j}];
        t.in_lo = lo;
        std::vector<int> in_mod, out_mod;
        for (int i = lo; i < hi; ++i) in_mod.push_back(i);
        for (int i = 0; i < l; ++i)
          if (i < lo || i >= hi) {
            out_mod.push_back(i);
            t.out_limb.push_back((uint16_t)i);
          }
        for (int k = 0; k < c->ks_k[l]; ++k) {
          out_mod.push_back(L + k);
          t.out_limb.push_back((uint16_t)(l + k));
        }
        for (int m : out_mod) t.out_pidx.push_back((uint8_t)m);
        add_table(t, in_mod, out_mod);
      }
    }
    // ModDown from the first k special primes to the q-limbs, per k in use
    for (int k = 1; k <= K; ++k) {
      if (!c->key_lmax[k]) continue;
      ConvTable& t = c->moddown[k];
      t.in_lo = L;
      std::vector<int> in_mod, out_mod;
      for (int kk = 0; kk < k; ++kk) in_mod.push_back(L + kk);
      for (int i = 0; i < L; ++i) {
        out_mod.push_back(i);
        t.out_limb.push_back((uint16_t)i);
        t.out_pidx.push_back((uint8_t)i);
      }
      add_table(t, in_mod, out_mod);
    }
    // relinearisation fused with rescale at level l: B' = {p_0..p_{K_l-1},
    // q_{l-1}} -> q_0..q_{l-2}
    for (int l = 2; l <= L; ++l) {
      ConvTable& t = c->fused[l];
      t.in_lo = 0;
      std::vector<int> in_mod, out_mod;
      for (int kk = 0; kk < c->ks_k[l]; ++kk) in_mod.push_back(L + kk);
      in_mod.push_back(l - 1);
      for (int m : in_mod) t.in_pidx.push_back((uint8_t)m);
      for (int i = 0; i < l - 1; ++i) {
        out_mod.push_back(i);
        t.out_limb.push_back((uint16_t)i);
        t.out_pidx.push_back((uint8_t)i);
      }
      add_table(t, in_mod, out_mod);
    }
    c->d_conv_store = upload(c.get(), store);
    for (auto& f : fix) f.first->dev = c->d_conv_store + f.second;
    // the scale pairs of every table's inputs (hinv N^-1 and ipsi[1] hinv
    // N^-1), and per level the ModUp digits' pairs in limb order
    {
      std::vector<ulonglong2> sc;
      std::vector<std::pair<ConvTable*, size_t>> sfix;
      auto pairs_of = [&](const ConvTable& t, size_t base) {
        for (int i = 0; i < t.n_in; ++i) {
          const int mi = t.in_pidx.empty() ? t.in_lo + i : t.in_pidx[i];
          const u64 q = c->mod[mi];
          const u64 a = host_mulmod(store[base + i], h_ninv[mi], q);
          const u64 b = host_mulmod(a, h_iw1[mi], q);
          sc.push_back(make_ulonglong2(a, shoup_companion(a, q)));
          sc.push_back(make_ulonglong2(b, shoup_companion(b, q)));
        }
      };
      for (auto& f : fix) {
        sfix.push_back({f.first, sc.size()});
        pairs_of(*f.first, f.second);
      }
      std::vector<size_t> mfix(L + 1, 0);
      for (int l = 1; l <= L; ++l) {
        mfix[l] = sc.size();
        const int beta = (l + alpha - 1) / alpha;
        for (int j = 0; j < beta; ++j)
          for (auto& f : fix)
            if (f.first == &c->modup[{l, j}]) pairs_of(*f.first, f.second);
      }
      c->d_iscale_store = upload(c.get(), sc);
      for (auto& f : sfix) f.first->iscale = c->d_iscale_store + f.second;
      for (int l = 1; l <= L; ++l) c->modup_iscale[l] = c->d_iscale_store + mfix[l];
    }
    // constants of the fused division by P' = P q_{l-1}, per level:
    // [P mod q_i, Shoup](i < l) [P'^-1 mod q_i, Shoup](i < l-1)
    // [-h mod q_i](i < l-1) [h (P'/m_j)^-1 mod m_j](j <= K_l), h = (P' - 1)/2
    // (the rounding offset, added to every coefficient inside the conversion)
    for (int l = 2; l <= L; ++l) {
      const int K_l = c->ks_k[l];
      std::vector<u64> fz;
      for (int i = 0; i < l; ++i) {
        const u64 q = c->mod[i];
        u64 Pm = 1;
        for (int kk = 0; kk < K_l; ++kk) Pm = host_mulmod(Pm, c->mod[L + kk] % q, q);
        fz.push_back(Pm);
        fz.push_back(shoup_companion(Pm, q));
      }
      std::vector<u64> hq;
      for (int i = 0; i < l - 1; ++i) {
        const u64 q = c->mod[i];
        u64 Pp = c->mod[l - 1] % q;
        for (int kk = 0; kk < K_l; ++kk) Pp = host_mulmod(Pp, c->mod[L + kk] % q, q);
        const u64 inv = host_inv(Pp, q);
        fz.push_back(inv);
        fz.push_back(shoup_companion(inv, q));
        const u64 h = host_mulmod((Pp + q - 1) % q, (q + 1) / 2, q);  // (P' - 1) / 2 mod q
        hq.push_back(h ? q - h : 0);
      }
      fz.insert(fz.end(), hq.begin(), hq.end());
      std::vector<u64> bm;
      for (int kk = 0; kk < K_l; ++kk) bm.push_back(c->mod[L + kk]);
      bm.push_back(c->mod[l - 1]);
      for (size_t jj = 0; jj < bm.size(); ++jj) {
        const u64 m = bm[jj];
        u64 r = 1;  // (P'/m_j) mod m_j
        for (size_t j2 = 0; j2 < bm.size(); ++j2)
          if (j2 != jj) r = host_mulmod(r, bm[j2] % m, m);
        fz.push_back(host_mulmod((m - 1) / 2, host_inv(r, m), m));  // h = -1/2 mod m_j
      }
      c->d_fused[l] = upload(c.get(), fz);
    }
    for (int k = 1; k <= K; ++k) {
      if (!c->key_lmax[k]) continue;
      std::vector<u64> pinv((size_t)L * 2);
      for (int i = 0; i < L; ++i) {
        const u64 q = c->mod[i];
        u64 Pm = 1;
        for (int kk = 0; kk < k; ++kk) Pm = host_mulmod(Pm, c->mod[L + kk] % q, q);
        pinv[2 * i] = host_inv(Pm, q);
        pinv[2 * i + 1] = shoup_companion(pinv[2 * i], q);
      }
      c->d_pinv[k] = upload(c.get(), pinv);
    }
  }
  // encoding tables
  {
    const int M = N / 2, logM = P.logN - 1;
    std::vector<double> W(M), T(2 * M);
    std::vector<double2> w2(M / 2), t2(M);
    auto pack = [&](void) {
      for (int t = 0; t < M / 2; ++t) w2[t] = make_double2(W[2 * t], W[2 * t + 1]);
      for (int k = 0; k < M; ++k) t2[k] = make_double2(T[2 * k], T[2 * k + 1]);
    };
    fft_twiddles(P.logN, -1, W.data(), T.data());
    {
      std::vector<longlong2> wq(M / 2), tq(M);
      for (int t = 0; t < M / 2; ++t)
        wq[t] = make_longlong2(std::llrint(std::ldexp(W[2 * t], 62)),
                               std::llrint(std::ldexp(W[2 * t + 1], 62)));
      for (int k = 0; k < M; ++k)
        tq[k] = make_longlong2(std::llrint(std::ldexp(T[2 * k], 62)),
                               std::llrint(std::ldexp(T[2 * k + 1], 62)));
      c->d_fftWq = upload(c.get(), wq);
      c->d_fftTq = upload(c.get(), tq);
    }
    fft_twiddles(P.logN, +1, W.data(), T.data());
    pack();
    c->d_fftW_dec = upload(c.get(), w2);
    c->d_fftT_dec = upload(c.get(), t2);
    std::vector<int> pos(M), uu(M);
    u64 g = 1;
    const u64 twoN = (u64)2 * N;
    for (int j = 0; j < M; ++j) {
      uu[j] = (int)((g - 1) / 4);
      pos[j] = bitrev_host(uu[j], logM);
      g = (g * 5) % twoN;
    }
    c->d_slot_u = upload(c.get(), uu);
    std::vector<int> inv(M);
    for (int j = 0; j < M; ++j) inv[pos[j]] = j;
    c->d_slot_inv = upload(c.get(), inv);
  }
  return c.release();
}

Context* ctx_child(const Context* base, cudaStream_t stream) {
  GWHE_REQUIRE(base && !base->parent, ST_EINVAL, "a child needs a root context");
  GWHE_REQUIRE(base->have_keys, ST_ENOKEY, "generate the keys before making child contexts");
  require_device(base);
  std::unique_ptr<Context> c(new Context(*base));
  c->parent = base;
  c->stream = stream;
  c->masks.clear();
  c->pin_stage[0] = c->pin_stage[1] = nullptr;  // staging buffers are per context
  c->pin_stage_bytes = 0;
  c->pin_state = nullptr;
  c->pin_state_bytes = 0;
  c->pin_state_lent = false;
  c->ks_count = 0;
  c->launches = 0;
  for (long& v : c->ks_by_level) v = 0;
  c->prof = Prof();
  c->last_error.clear();
  return c.release();
}

int device_check(int context_device, int current_device) {
  return (context_device >= 0 && current_device == context_device) ? ST_OK : ST_EINVAL;
}

void require_device(const Context* c) {
  int cur = -1;
  GWHE_CUDA(cudaGetDevice(&cur));
  if (device_check(c->device, cur) != ST_OK)
    throw Error(ST_EINVAL, "the current CUDA device (" + std::to_string(cur) +
                               ") is not the context's device (" + std::to_string(c->device) + ")");
}

// releases the context's memory on its own device and restores the caller's
static void ctx_destroy_on_device(Context* c);
void ctx_destroy(Context* c) {
  if (!c) return;
  int cur = -1;
  const bool have = cudaGetDevice(&cur) == cudaSuccess;
  if (have && cur != c->device) cudaSetDevice(c->device);
  ctx_destroy_on_device(c);
  if (have && cur != c->device) cudaSetDevice(cur);
}

static void ctx_destroy_on_device(Context* c) {
  cudaStreamSynchronize(c->stream);
  for (void* p : c->pin_stage)
    if (p) cudaFreeHost(p);
  if (c->pin_state) cudaFreeHost(c->pin_state);
  if (c->parent) {  // only the child's own state
    for (auto& kv : c->masks) {
      cudaFreeAsync(kv.second.pt, c->stream);
      cudaEventDestroy(kv.second.done);
    }
    for (auto& r : c->prof.recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    delete c;
    return;
  }
  for (void* p : {(void*)c->d_psiB, (void*)c->d_ipsiB}) if (p) cudaFree(p);
  for (void* p : {(void*)c->d_mod, (void*)c->d_psi, (void*)c->d_ipsi, (void*)c->d_ninv, (void*)c->d_ninv_sh, (void*)c->d_iw1n, (void*)c->d_iscale_store, (void*)c->d_rescale,
                  (void*)c->d_conv_store, (void*)c->d_fftW_dec, (void*)c->d_fftT_dec,
                  (void*)c->d_fftWq, (void*)c->d_fftTq,
                  (void*)c->d_slot_u, (void*)c->d_slot_inv})
    if (p) cudaFree(p);
  for (auto& kv : c->masks) {
      cudaFreeAsync(kv.second.pt, c->stream);
      cudaEventDestroy(kv.second.done);
    }
  for (u64* p : c->d_pinv)
    if (p) cudaFree(p);
  for (u64* p : c->d_fused)
    if (p) cudaFree(p);
  for (auto& r : c->prof.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  if (c->d_sk) cudaFreeAsync(c->d_sk, c->stream);
  if (c->d_pk) cudaFreeAsync(c->d_pk, c->stream);
  for (auto& kv : c->ksk)
    for (const Ksk& f : kv.second.fam)
      if (f.d) cudaFreeAsync(f.d, c->stream);
  cudaStreamSynchronize(c->stream);
  delete c;
}

// ---------------------------------------------------------------- keys
static RowMap rows_all(const Context* c, int first, int count, int poly_stride, int npoly) {
  RowMap rm;
  rm.npoly = npoly;
  rm.nl = count;
  rm.poly_stride = poly_stride;
  for (int i = 0; i < count; ++i) {
    rm.off[i] = (uint16_t)i;
    rm.pidx[i] = (uint8_t)(first + i);
  }
  return rm;
}

const Ksk& key_family(const Context* c, u32 key_id, int l) {
  auto it = c->ksk.find(key_id);
  GWHE_REQUIRE(it != c->ksk.end(), ST_ENOKEY, "missing switching key " + std::to_string(key_id));
  GWHE_REQUIRE(l >= 1 && l <= c->P.L, ST_EINVAL, "bad level for a key switch");
  const Ksk& f = it->second.fam[c->ks_k[l]];
  GWHE_REQUIRE(f.d && f.lmax >= l, ST_ENOKEY, "switching key family missing");
  return f;
}

// target: residues of the key's target over all L + K moduli ([L+K][N], NTT
// domain).  One family per special-prime count k in use: digit j of family k
// holds b_j = -a_j s + e_j + [u in digit j] P_k t and a_j, rows q_0..q_{lmax-1},
// p_0..p_{k-1}; the random streams are keyed by (key id, k, j) and the uniform
// rows by the global modulus index.
static void make_ksk(Context* c, u32 key_id, const u64* target) {
  const int N = c->N, L = c->P.L, K = c->P.K;
  KeySet ks;
  for (int k = 1; k <= K; ++k) {
    const int lmax = c->key_lmax[k];
    if (!lmax) continue;
    Ksk f;
    f.k = k;
    f.lmax = lmax;
    f.dk = (lmax + c->alpha - 1) / c->alpha;
    const int nm = f.rows();
    f.d = dalloc_u64(c, (size_t)f.dk * 2 * nm * N);
    std::vector<uint8_t> pidx(nm);
    std::vector<int> gm(nm);
    for (int u = 0; u < nm; ++u) {
      gm[u] = u < lmax ? u : L + (u - lmax);
      pidx[u] = (uint8_t)gm[u];
    }
    RowMap rm;
    rm.npoly = 1;
    rm.nl = nm;
    rm.poly_stride = nm;
    for (int u = 0; u < nm; ++u) {
      rm.off[u] = (uint16_t)u;
      rm.pidx[u] = pidx[u];
    }
    Tmp e(c, sizeof(u64) * nm * N);
    for (int j = 0; j < f.dk; ++j) {
      u64* bj = f.d + ((size_t)j * 2 + 0) * nm * N;
      u64* aj = f.d + ((size_t)j * 2 + 1) * nm * N;
      sample_cbd_rns(c, obj_ksk_e(key_id, k, j), e.u(), pidx.data(), nm);
      ntt_forward(c, e.u(), rm);
      for (int u = 0; u < nm; ++u)
        sample_uniform(c, obj_ksk_a(key_id, k, j), (u32)gm[u], gm[u], aj + (size_t)u * N);
      ntt_forward(c, aj, rm);
      const int lo = j * c->alpha, hi = std::min(lo + c->alpha, lmax);
      for (int u = 0; u < nm; ++u) {
        u64 pm = 0;
        const u64* t = nullptr;
        const u64 m = c->mod[gm[u]];
        if (u >= lo && u < hi) {
          pm = 1;
          for (int kk = 0; kk < k; ++kk) pm = host_mulmod(pm, c->mod[L + kk] % m, m);
          t = target + (size_t)gm[u] * N;
        }
        ksk_combine(c, bj + (size_t)u * N, aj + (size_t)u * N, e.u() + (size_t)u * N,
                    c->d_sk + (size_t)gm[u] * N, t, pm, gm[u]);
      }
    }
    ks.fam[k] = f;
  }
  auto it = c->ksk.find(key_id);
  if (it != c->ksk.end())
    for (const Ksk& f : it->second.fam)
      if (f.d) dfree(c, f.d);
  c->ksk[key_id] = ks;
}

void add_galois_key(Context* c, u32 g) {
  GWHE_REQUIRE(!c->parent, ST_EINVAL, "keys are generated on the root context");
  const int N = c->N, nm = c->nmod;
  Tmp t(c, sizeof(u64) * nm * N);
  automorph_ntt(c, PolyView{t.u(), nm}, CPolyView{c->d_sk, nm}, 1, nm, g);
  make_ksk(c, g, t.u());
}

void keygen(Context* c, const std::vector<u32>& galois) {
  GWHE_REQUIRE(!c->parent, ST_EINVAL, "keys are generated on the root context");
  const int N = c->N, L = c->P.L, nm = c->nmod;
  std::vector<uint8_t> pidx(nm);
  for (int u = 0; u < nm; ++u) pidx[u] = (uint8_t)u;
  if (!c->d_sk) c->d_sk = dalloc_u64(c, (size_t)nm * N);
  sample_ternary_rns(c, kObjSk, c->d_sk, pidx.data(), nm);
  ntt_forward(c, c->d_sk, rows_all(c, 0, nm, nm, 1));
  if (!c->d_pk) c->d_pk = dalloc_u64(c, (size_t)2 * L * N);
  {
    Tmp e(c, sizeof(u64) * L * N);
    sample_cbd_rns(c, kObjPkE, e.u(), pidx.data(), L);
    ntt_forward(c, e.u(), rows_all(c, 0, L, L, 1));
    u64* a = c->d_pk + (size_t)L * N;
    for (int i = 0; i < L; ++i) sample_uniform(c, kObjPkA, (u32)i, i, a + (size_t)i * N);
    ntt_forward(c, a, rows_all(c, 0, L, L, 1));
    for (int i = 0; i < L; ++i)
      ksk_combine(c, c->d_pk + (size_t)i * N, a + (size_t)i * N, e.u() + (size_t)i * N,
                  c->d_sk + (size_t)i * N, nullptr, 0, i);
  }
  {
    // relinearisation: target s^2 (limb u of the secret lies modulo mod[u])
    Tmp s2(c, sizeof(u64) * nm * N);
    ew_mul_plain(c, PolyView{s2.u(), nm}, CPolyView{c->d_sk, nm}, 1, nm, c->d_sk);
    make_ksk(c, 0, s2.u());
  }
  for (u32 g : galois) add_galois_key(c, g);
  c->have_keys = true;
}

u32 galois_for_rotation(const Context* c, int r) {
  const int M = c->N / 2;
  const u64 twoN = (u64)2 * c->N;
  int e = ((r % M) + M) % M;
  u64 g = 1;
  for (int i = 0; i < e; ++i) g = (g * 5) % twoN;
  return (u32)g;
}
u32 galois_conj(const Context* c) { return (u32)(2 * c->N - 1); }

// ---------------------------------------------------------------- arithmetic
static void check_scales(double a, double b) {
  if (std::fabs(a / b - 1.0) > std::ldexp(1.0, -10))
    throw Error(ST_ESCALE, "scale mismatch: " + std::to_string(a) + " vs " + std::to_string(b));
}

void op_addsub(Context* c, const Ct& a, const Ct& b, Ct& out, bool sub) {
  GWHE_REQUIRE(a.l == b.l && a.npoly == b.npoly, ST_ELEVEL, "operands at different levels");
  GWHE_REQUIRE(out.cap >= a.l && out.npoly == a.npoly, ST_EINVAL, "output too small");
  check_scales(a.scale, b.scale);
  ew_addsub(c, pv(out), cpv(a), cpv(b), a.npoly, a.l, sub);
  out.l = a.l;
  out.scale = a.scale;
}

void op_negate(Context* c, const Ct& a, Ct& out) {
  ew_negate(c, pv(out), cpv(a), a.npoly, a.l);
  out.l = a.l;
  out.scale = a.scale;
}

static std::vector<u64> signed_residues(const Context* c, i64 v, int l) {
  std::vector<u64> r(l);
  for (int i = 0; i < l; ++i) {
    const u64 q = c->mod[i];
    if (v >= 0) {
      r[i] = (u64)v % q;
    } else {
      const u64 t = ((u64)(-(v + 1)) + 1) % q;
      r[i] = t ? q - t : 0;
    }
  }
  return r;
}

void op_add_const(Context* c, Ct& ct, double v) {
  const i64 m0 = std::llrint(v * ct.scale);
  const std::vector<u64> r = signed_residues(c, m0, ct.l);
  ew_add_scalar_poly0(c, pv(ct), ct.l, r.data());
}

void op_mul_int(Context* c, Ct& ct, i64 k) {
  const std::vector<u64> r = signed_residues(c, k, ct.l);
  ew_mul_scalar(c, pv(ct), cpv(ct), ct.npoly, ct.l, r.data());
}

void op_mul_const(Context* c, Ct& ct, double v) {
  GWHE_REQUIRE(ct.l >= 2, ST_ELEVEL, "no level left for a constant product");
  const u64 ql = c->mod[ct.l - 1];
  const i64 m0 = std::llrint(v * (double)ql);
  const std::vector<u64> r = signed_residues(c, m0, ct.l);
  ew_mul_scalar(c, pv(ct), cpv(ct), ct.npoly, ct.l, r.data());
  ct.scale = ct.scale * (double)ql;
  op_rescale(c, ct);
}

void op_mul_plain(Context* c, const Ct& a, const u64* pt, double pt_scale, Ct& out) {
  ew_mul_plain(c, pv(out), cpv(a), a.npoly, a.l, pt);
  out.l = a.l;
  out.scale = a.scale * pt_scale;
}

void op_add_plain(Context* c, Ct& ct, const u64* pt) { ew_add_plain_poly0(c, pv(ct), ct.l, pt); }

void op_tensor_mac(Context* c, const std::vector<std::pair<const Ct*, const Ct*>>& terms, Ct& out3) {
  GWHE_REQUIRE(!terms.empty(), ST_EINVAL, "empty tensor sum");
  const int l = terms[0].first->l;
  std::vector<MacPair> hp;
  for (auto& t : terms) {
    GWHE_REQUIRE(t.first->l == l && t.second->l == l, ST_ELEVEL, "tensor operands at different levels");
    check_scales(t.first->scale * t.second->scale,
                 terms[0].first->scale * terms[0].second->scale);
    hp.push_back(MacPair{t.first->d, t.second->d, t.first->cap, t.second->cap});
  }
  Tmp dp(c, sizeof(MacPair) * hp.size());
  GWHE_CUDA(cudaMemcpyAsync(dp.p, hp.data(), sizeof(MacPair) * hp.size(), cudaMemcpyHostToDevice,
                            c->stream));
  GWHE_REQUIRE(out3.npoly == 3 && out3.cap >= l, ST_EINVAL, "tensor output too small");
  tensor_mac_set(c, pv(out3), 0, dp.as<MacPair>(), (int)hp.size(), 1, l);
  out3.l = l;
  out3.scale = terms[0].first->scale * terms[0].second->scale;
}

void keyswitch(Context* c, const u64* x_ntt, int l, const KeySet& key, u64* out0, u64* out1,
               const u64* add0, const u64* add1) {
  keyswitch_set(c, x_ntt, 0, 1, l, key, out0, out1, 0, add0, add1, 0, 0);
}

void op_relin(Context* c, const Ct& t3, Ct& out) {
  GWHE_REQUIRE(t3.npoly == 3, ST_EINVAL, "relinearisation needs a tensor");
  auto it = c->ksk.find(0);
  GWHE_REQUIRE(it != c->ksk.end(), ST_ENOKEY, "no relinearisation key");
  const int l = t3.l;
  GWHE_REQUIRE(out.cap >= l && out.npoly == 2, ST_EINVAL, "output too small");
  keyswitch(c, t3.poly(2), l, it->second, out.poly(0), out.poly(1), t3.poly(0), t3.poly(1));
  out.l = l;
  out.scale = t3.scale;
}

void op_rescale(Context* c, Ct& ct) {
  const int l = ct.l, np = ct.npoly, N = c->N;
  GWHE_REQUIRE(l >= 2, ST_ELEVEL, "no level left to rescale");
  Tmp last(c, sizeof(u64) * np * N);
  GWHE_CUDA(cudaMemcpy2DAsync(last.p, sizeof(u64) * N, ct.limb(0, l - 1),
                              sizeof(u64) * (size_t)ct.cap * N, sizeof(u64) * N, np,
                              cudaMemcpyDeviceToDevice, c->stream));
  RowMap rl;
  rl.npoly = np;
  rl.nl = 1;
  rl.poly_stride = 1;
  rl.off[0] = 0;
  rl.pidx[0] = (uint8_t)(l - 1);
  ntt_inverse(c, last.u(), rl);
  Tmp tmp(c, sizeof(u64) * np * (l - 1) * N);
  rescale_prep(c, last.u(), np, l, tmp.u());
  ntt_forward(c, tmp.u(), rows_q(np, l - 1, l - 1));
  rescale_combine(c, pv(ct), tmp.u(), np, l);
  ct.l = l - 1;
  ct.scale = ct.scale / (double)c->mod[l - 1];
}

void op_mult(Context* c, const Ct& a, const Ct& b, Ct& out) {
  GWHE_REQUIRE(a.l == b.l, ST_ELEVEL, "operands at different levels");
  CtPtr t = ct_new(c, 3, a.l, a.l, 1.0);
  op_tensor_mac(c, {{&a, &b}}, *t);
  op_relin_rescale(c, *t, out);
}

void op_galois(Context* c, const Ct& a, u32 g, Ct& out) {
  auto it = c->ksk.find(g);
  GWHE_REQUIRE(it != c->ksk.end(), ST_ENOKEY, "missing Galois key " + std::to_string(g));
  GWHE_REQUIRE(&a != &out && a.d != out.d, ST_EINVAL, "automorphism output must not alias");
  GWHE_REQUIRE(out.cap >= a.l, ST_EINVAL, "output too small");
  const int l = a.l;
  automorph_ntt(c, pv(out), cpv(a), 2, l, g);
  keyswitch(c, out.poly(1), l, it->second, out.poly(0), out.poly(1), out.poly(0), nullptr);
  out.l = l;
  out.scale = a.scale;
}

void op_rotate(Context* c, const Ct& a, int r, Ct& out) { op_galois(c, a, galois_for_rotation(c, r), out); }
void op_conj(Context* c, const Ct& a, Ct& out) { op_galois(c, a, galois_conj(c), out); }

void op_drop(Ct& ct, int l) {
  GWHE_REQUIRE(l >= 1 && l <= ct.l, ST_ELEVEL, "cannot raise a level");
  ct.l = l;
}

// ---------------------------------------------------------------- sets
CtSet::~CtSet() {
  if (owned && d && ctx) dfree(ctx, d);
}

CtSet CtSet::slice(int first, int n, int lv) const {
  GWHE_REQUIRE(first >= 0 && n >= 1 && first + n <= cnt && lv <= l, ST_EINVAL, "bad set slice");
  CtSet v;
  v.ctx = ctx;
  v.d = item(first);
  v.cnt = n;
  v.npoly = npoly;
  v.cap = cap;
  v.l = lv;
  v.scale = scale;
  v.owned = false;
  return v;
}

CtPtr CtSet::view(int i) const {
  CtPtr v(new Ct());
  v->ctx = ctx;
  v->d = item(i);
  v->npoly = npoly;
  v->cap = cap;
  v->l = l;
  v->scale = scale;
  v->owned = false;
  return v;
}

Ct CtSet::all() const {
  Ct v;
  v.ctx = ctx;
  v.d = d;
  v.npoly = npoly * cnt;
  v.cap = cap;
  v.l = l;
  v.scale = scale;
  v.owned = false;
  return v;
}

CtSetPtr set_new(Context* c, int cnt, int npoly, int cap, int l, double scale) {
  GWHE_REQUIRE(cnt >= 1 && l <= cap, ST_EINVAL, "bad ciphertext set");
  CtSetPtr s(new CtSet());
  s->ctx = c;
  s->cnt = cnt;
  s->npoly = npoly;
  s->cap = cap;
  s->l = l;
  s->scale = scale;
  s->d = dalloc_u64(c, (size_t)cnt * npoly * cap * c->N);
  return s;
}

template <class T>
static T* upload_async(Context* c, Tmp& t, const std::vector<T>& v) {
  GWHE_CUDA(cudaMemcpyAsync(t.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice,
                            c->stream));
  return t.as<T>();
}

// ModUp of cnt inputs (NTT domain, item i at x + i x_stride, l limbs): the
// coefficient form of each digit is converted to the other limbs of the
// extended basis (K = ks_k[l] special primes) and transformed back; ext is
// [cnt][beta][ne][N] and omits the digit's own limbs (read from x).
static void modup_ext(Context* c, const u64* x, size_t x_stride, int cnt, int l, u64* ext) {
  const size_t N = c->N;
  const int ne = l + c->ks_k[l];
  const int beta = (l + c->alpha - 1) / c->alpha;
  Tmp xc(c, sizeof(u64) * cnt * l * N);
  GWHE_CUDA(cudaMemcpy2DAsync(xc.p, sizeof(u64) * l * N, x,
                              sizeof(u64) * std::max<size_t>(x_stride, l * N), sizeof(u64) * l * N,
                              cnt, cudaMemcpyDeviceToDevice, c->stream));
  // the coefficient form of every digit limb times its conversion's hinv
  const ulonglong2* isc = c->modup_iscale[l];
  ntt_inverse(c, xc.u(), rows_q(cnt, l, l), isc);
  modup_convert_set(c, xc.u(), l, ext, cnt, isc != nullptr);
  // the new limbs of every digit in one transform launch
  RowMap rm;
  rm.npoly = cnt;
  rm.nl = 0;
  rm.poly_stride = beta * ne;
  for (int j = 0; j < beta; ++j) {
    const ConvTable& t = c->modup.at({l, j});
    GWHE_REQUIRE(rm.nl + t.n_out <= kMaxRowMap, ST_EINVAL, "ModUp rows exceed a row map");
    for (int o = 0; o < t.n_out; ++o, ++rm.nl) {
      rm.off[rm.nl] = (uint16_t)(j * ne + t.out_limb[o]);
      rm.pidx[rm.nl] = t.out_pidx[o];
    }
  }
  ntt_forward(c, ext, rm);
}

// ModDown of cnt key products acc ([cnt][2][ne][N], NTT domain) by P_K into
// out0/out1 (+ add0/add1), item strides as given.
static void moddown_out(Context* c, u64* acc, int cnt, int l, int K, u64* out0, u64* out1,
                        size_t o_stride, const u64* add0, const u64* add1, size_t a0_stride,
                        size_t a1_stride) {
  const size_t N = c->N;
  const int L = c->P.L, ne = l + K;
  RowMap rk;
  rk.npoly = 2 * cnt;
  rk.nl = K;
  rk.poly_stride = ne;
  for (int k = 0; k < K; ++k) {
    rk.off[k] = (uint16_t)(l + k);
    rk.pidx[k] = (uint8_t)(L + k);
  }
  const ulonglong2* isc = c->moddown[K].iscale;  // the conversion's hinv, merged
  ntt_inverse(c, acc, rk, isc);
  Tmp conv(c, sizeof(u64) * cnt * 2 * l * N);
  moddown_convert_set(c, acc, l, K, conv.u(), cnt, isc != nullptr);
  // the transform's row pass ends with (acc - NTT(conv)) P^-1 + add
  const MdEpi epi{acc, l, K, out0, out1, o_stride, add0, add1, a0_stride, a1_stride, c->d_pinv[K]};
  if (ntt_forward_moddown(c, conv.u(), cnt, epi)) return;
  ntt_forward(c, conv.u(), rows_q(2 * cnt, l, l));
  moddown_combine_set(c, acc, conv.u(), l, K, cnt, out0, out1, o_stride, add0, add1, a0_stride,
                      a1_stride);
}

// Hybrid key switch of cnt ciphertext parts at level l with the key family of
// K_l special primes: ModUp (iNTT, fast base conversion per digit, NTT of the
// new limbs), the inner product with the key digits, ModDown (iNTT of the
// special limbs, conversion to the q-limbs, NTT, (x - conv) P_{K_l}^-1).
void keyswitch_set(Context* c, const u64* x, size_t x_stride, int cnt, int l, const KeySet& key,
                   u64* out0, u64* out1, size_t o_stride, const u64* add0, const u64* add1,
                   size_t a0_stride, size_t a1_stride) {
  const size_t N = c->N;
  const Ksk& fam = key.fam[c->ks_k[l]];
  GWHE_REQUIRE(fam.d && fam.lmax >= l, ST_ENOKEY, "switching key family missing");
  const int K = fam.k, ne = l + K;
  const int beta = (l + c->alpha - 1) / c->alpha;
  c->ks_count += cnt;
  c->ks_by_level[l] += cnt;
  Tmp ext(c, sizeof(u64) * cnt * beta * ne * N);
  modup_ext(c, x, x_stride, cnt, l, ext.u());
  Tmp acc(c, sizeof(u64) * cnt * 2 * ne * N);
  ks_inner_set(c, x, x_stride, l, ext.u(), fam, acc.u(), cnt);
  moddown_out(c, acc.u(), cnt, l, K, out0, out1, o_stride, add0, add1, a0_stride, a1_stride);
}

// s[i] <- s[i] + sum_{r in rs} Rotate(s[i], r), the rotations' key switches
// hoisted: one ModUp of each c1, the automorphisms applied to the ModUp
// digits, the inner products with the rotations' keys summed in the extended
// basis, one ModDown; c0 + sum_r sigma_r(c0) is added exactly.  Counts as one
// key switch per item.
void set_rotate_sum(Context* c, CtSet& s, const std::vector<int>& rs) {
  const size_t N = c->N;
  const int l = s.l, cnt = s.cnt;
  GWHE_REQUIRE(!rs.empty() && (int)rs.size() <= kMaxHoist, ST_EINVAL, "bad hoisted rotation set");
  const int K = c->ks_k[l], ne = l + K;
  const int beta = (l + c->alpha - 1) / c->alpha;
  HoistKeys hk;
  hk.G = (int)rs.size();
  int key_lmax = 0;
  for (int g = 0; g < hk.G; ++g) {
    const u32 gal = galois_for_rotation(c, rs[g]);
    const Ksk& fam = key_family(c, gal, l);
    hk.key[g] = fam.d;
    hk.g[g] = gal;
    key_lmax = fam.lmax;
  }
  c->ks_count += cnt;
  c->ks_by_level[l] += cnt;
  u64* c1 = s.d + (size_t)s.cap * N;
  Tmp ext(c, sizeof(u64) * cnt * beta * ne * N);
  modup_ext(c, c1, s.stride(), cnt, l, ext.u());
  Tmp acc(c, sizeof(u64) * cnt * 2 * ne * N);
  ks_inner_hoist_set(c, c1, s.stride(), l, ext.u(), hk, key_lmax, K, acc.u(), cnt);
  Tmp t0(c, sizeof(u64) * cnt * l * N);
  automorph_sum_set(c, s.d, s.cap, s.stride(), t0.u(), l, cnt, hk);
  moddown_out(c, acc.u(), cnt, l, K, s.d, c1, s.stride(), t0.u(), c1, (size_t)l * N, s.stride());
}

std::vector<std::vector<int>> ladder_groups(const std::vector<int>& steps, int group) {
  // up to `group` consecutive doubling steps r, 2r, 4r, ... of a ladder
  // merge into one hoisted step over the rotations r, 2r, ..., (2^m - 1) r
  // (the same sum of rotations)
  GWHE_REQUIRE(group >= 1 && (1 << group) - 1 <= kMaxHoist, ST_EINVAL, "ladder group too long");
  std::vector<std::vector<int>> out;
  for (size_t i = 0; i < steps.size();) {
    size_t m = 1;
    while (m < (size_t)group && i + m < steps.size() && steps[i + m] == 2 * steps[i + m - 1])
      ++m;
    std::vector<int> g;
    for (int t = 1; t < (1 << m); ++t) g.push_back(t * steps[i]);
    out.push_back(g);
    i += m;
  }
  return out;
}

void set_ladder(Context* c, CtSet& s, const std::vector<int>& steps, int group) {
  GWHE_REQUIRE(s.npoly == 2, ST_EINVAL, "ladder needs ciphertexts");
  for (const auto& rs : ladder_groups(steps, group)) set_rotate_sum(c, s, rs);
}

void set_galois(Context* c, const CtSet& a, u32 g, CtSet& out) {
  auto it = c->ksk.find(g);
  GWHE_REQUIRE(it != c->ksk.end(), ST_ENOKEY, "missing Galois key " + std::to_string(g));
  GWHE_REQUIRE(out.cnt == a.cnt && out.cap >= a.l && a.d != out.d, ST_EINVAL, "bad galois set");
  const size_t N = c->N;
  const int l = a.l;
  Ct ai = a.all(), oi = out.all();
  automorph_ntt(c, PolyView{oi.d, oi.cap}, CPolyView{ai.d, ai.cap}, 2 * a.cnt, l, g);
  keyswitch_set(c, out.d + (size_t)out.cap * N, out.stride(), a.cnt, l, it->second, out.d,
                out.d + (size_t)out.cap * N, out.stride(), out.d, nullptr, out.stride(), 0);
  out.l = l;
  out.scale = a.scale;
}

void set_mask(Context* c, const std::vector<MaskItem>& items, double src_scale, double pt_scale,
              CtSet& out, bool rescale) {
  GWHE_REQUIRE((int)items.size() == out.cnt, ST_EINVAL, "mask set size");
  Tmp d(c, sizeof(MaskItem) * items.size());
  mask_set(c, upload_async(c, d, items), out.cnt, out.d, out.cap, out.stride(), out.l);
  out.scale = src_scale * pt_scale;
  if (rescale) set_rescale(c, out);
}

void set_tensor_mac(Context* c, const std::vector<std::pair<const Ct*, const Ct*>>& pairs,
                    int npairs, CtSet& out3, bool accumulate) {
  GWHE_REQUIRE(out3.npoly == 3 && (int)pairs.size() == npairs * out3.cnt, ST_EINVAL,
               "tensor set shape");
  const int l = pairs[0].first->l;
  std::vector<MacPair> hp;
  const double sc = pairs[0].first->scale * pairs[0].second->scale;
  for (auto& pr : pairs) {
    GWHE_REQUIRE(pr.first->l == l && pr.second->l == l, ST_ELEVEL,
                 "tensor operands at different levels");
    check_scales(pr.first->scale * pr.second->scale, sc);
    hp.push_back(MacPair{pr.first->d, pr.second->d, pr.first->cap, pr.second->cap});
  }
  GWHE_REQUIRE(out3.cap >= l, ST_EINVAL, "tensor output too small");
  if (accumulate) {
    GWHE_REQUIRE(out3.l == l, ST_ELEVEL, "accumulated tensor at another level");
    check_scales(out3.scale, sc);
  }
  Tmp d(c, sizeof(MacPair) * hp.size());
  tensor_mac_set(c, PolyView{out3.d, out3.cap}, out3.stride(), upload_async(c, d, hp), npairs,
                 out3.cnt, l, accumulate);
  out3.l = l;
  out3.scale = sc;
}

void set_relin(Context* c, const CtSet& t3, CtSet& out) {
  GWHE_REQUIRE(t3.npoly == 3 && out.npoly == 2 && out.cnt == t3.cnt && out.cap >= t3.l,
               ST_EINVAL, "relinearisation set shape");
  auto it = c->ksk.find(0);
  GWHE_REQUIRE(it != c->ksk.end(), ST_ENOKEY, "no relinearisation key");
  const size_t N = c->N;
  keyswitch_set(c, t3.d + (size_t)2 * t3.cap * N, t3.stride(), t3.cnt, t3.l, it->second, out.d,
                out.d + (size_t)out.cap * N, out.stride(), t3.d, t3.d + (size_t)t3.cap * N,
                t3.stride(), t3.stride());
  out.l = t3.l;
  out.scale = t3.scale;
}

void set_rescale(Context* c, CtSet& s) {
  Ct all = s.all();
  op_rescale(c, all);
  s.l = all.l;
  s.scale = all.scale;
}

// Relinearisation fused with the rescale after it, for cnt tensors at level l
// (item i at t3 + i t3_stride, cap t3_cap; NTT domain) into out (level
// l - 1): ModUp of d2 and the key product acc as in a key switch, then
// y = acc + P (d0, d1) divided once by P' = P q_{l-1}, rounding to nearest:
// the B' = {p_0..p_{K-1}, q_{l-1}} rows of y + floor(P'/2) back to the
// coefficient domain, their fast conversion to q_0..q_{l-2}, its NTT, and
// (y + floor(P'/2) - conv) P'^-1.
static void relin_rescale_items(Context* c, const u64* t3, size_t t3_stride, int t3_cap, int cnt,
                                int l, u64* out, size_t o_stride, int o_cap) {
  GWHE_REQUIRE(l >= 2, ST_ELEVEL, "no level left to rescale");
  const size_t N = c->N;
  const Ksk& fam = key_family(c, 0, l);
  const int K = fam.k, L = c->P.L, ne = l + K;
  const int beta = (l + c->alpha - 1) / c->alpha;
  c->ks_count += cnt;
  c->ks_by_level[l] += cnt;
  const u64* d2 = t3 + (size_t)2 * t3_cap * N;
  Tmp ext(c, sizeof(u64) * cnt * beta * ne * N);
  modup_ext(c, d2, t3_stride, cnt, l, ext.u());
  Tmp acc(c, sizeof(u64) * cnt * 2 * ne * N);
  ks_inner_set(c, d2, t3_stride, l, ext.u(), fam, acc.u(), cnt);
  Tmp bp(c, sizeof(u64) * cnt * 2 * (K + 1) * N);
  fused_prep_set(c, acc.u(), t3, t3_stride, t3_cap, bp.u(), l, K, cnt);
  RowMap rb;
  rb.npoly = 2 * cnt;
  rb.nl = K + 1;
  rb.poly_stride = K + 1;
  for (int j = 0; j <= K; ++j) {
    rb.off[j] = (uint16_t)j;
    rb.pidx[j] = (uint8_t)(j < K ? L + j : l - 1);
  }
  const ulonglong2* isc = c->fused[l].iscale;  // the conversion's hinv, merged
  ntt_inverse(c, bp.u(), rb, isc);
  Tmp conv(c, sizeof(u64) * cnt * 2 * (l - 1) * N);
  fused_convert_set(c, bp.u(), l, K, conv.u(), cnt, isc != nullptr);
  ntt_forward(c, conv.u(), rows_q(2 * cnt, l - 1, l - 1));
  fused_combine_set(c, acc.u(), t3, t3_stride, t3_cap, conv.u(), out, o_stride, o_cap, l, K, cnt);
}

void set_relin_rescale(Context* c, const CtSet& t3, CtSet& out) {
  GWHE_REQUIRE(t3.npoly == 3 && out.npoly == 2 && out.cnt == t3.cnt && out.cap >= t3.l - 1,
               ST_EINVAL, "relinearisation set shape");
  GWHE_REQUIRE(out.d != t3.d, ST_EINVAL, "fused relinearisation output must not alias");
  relin_rescale_items(c, t3.d, t3.stride(), t3.cap, t3.cnt, t3.l, out.d, out.stride(), out.cap);
  out.l = t3.l - 1;
  out.scale = t3.scale / (double)c->mod[t3.l - 1];
}

void op_relin_rescale(Context* c, const Ct& t3, Ct& out) {
  GWHE_REQUIRE(t3.npoly == 3 && out.npoly == 2 && out.cap >= t3.l - 1, ST_EINVAL,
               "relinearisation needs a tensor");
  GWHE_REQUIRE(out.d != t3.d, ST_EINVAL, "fused relinearisation output must not alias");
  relin_rescale_items(c, t3.d, 0, t3.cap, 1, t3.l, out.d, 0, out.cap);
  out.l = t3.l - 1;
  out.scale = t3.scale / (double)c->mod[t3.l - 1];
}

void set_mult(Context* c, const std::vector<std::pair<const Ct*, const Ct*>>& pairs, CtSet& out) {
  const int l = pairs[0].first->l;
  CtSetPtr t3 = set_new(c, out.cnt, 3, l, l, 1.0);
  set_tensor_mac(c, pairs, 1, *t3);
  set_relin_rescale(c, *t3, out);
}

// ---------------------------------------------------------------- encoding
void encode_to_ntt(Context* c, const double2* z, int count, double scale, int l, u64* pt) {
  const int N = c->N;
  Tmp work(c, sizeof(double2) * count * (N / 2));
  Tmp ints(c, sizeof(i64) * count * N);
  encode_batch(c, z, count, scale, ints.as<i64>(), work.as<double2>());
  int_to_rns(c, ints.as<i64>(), count, l, pt);
  ntt_forward(c, pt, rows_q(count, l, l));
}

const u64* mask_pt(Context* c, int kind, long index, int l, double scale,
                   const std::vector<double2>& slots) {
  auto key = std::make_tuple(kind, index, l, scale);
  auto it = c->masks.find(key);
  if (it != c->masks.end()) {
    // encoded on another stream of this context (a concurrent chain of the
    // covariate phase): this stream waits for the encoding
    if (it->second.stream != c->stream)
      GWHE_CUDA(cudaStreamWaitEvent(c->stream, it->second.done, 0));
    return it->second.pt;
  }
  const int M = c->N / 2;
  GWHE_REQUIRE((int)slots.size() == M, ST_EINVAL, "mask must hold N/2 slots");
  Tmp z(c, sizeof(double2) * M);
  GWHE_CUDA(cudaMemcpyAsync(z.p, slots.data(), sizeof(double2) * M, cudaMemcpyHostToDevice,
                            c->stream));
  // from the stream-ordered pool and without a host wait: later launches on
  // this stream are ordered after the encoding, other streams wait for the
  // event
  u64* pt = dalloc_u64(c, (size_t)l * c->N);
  encode_to_ntt(c, z.as<double2>(), 1, scale, l, pt);
  cudaEvent_t done;
  GWHE_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
  GWHE_CUDA(cudaEventRecord(done, c->stream));
  c->masks[key] = Context::Mask{pt, c->stream, done};
  return pt;
}

void encrypt_coeffs(Context* c, const i64* m, int count, int l, u64 id0, u64* out, int out_cap,
                    const u64* d_ids) {
  GWHE_REQUIRE(c->d_pk, ST_ENOKEY, "no public key");
  const int N = c->N;
  Tmp tmp(c, sizeof(u64) * count * 3 * l * N);
  enc_sample(c, id0, count, l, m, tmp.u(), d_ids);
  ntt_forward(c, tmp.u(), rows_q(count * 3, l, l));
  enc_combine(c, tmp.u(), count, l, out, out_cap, (size_t)2 * out_cap * N);
}

void encrypt_slots(Context* c, const double2* z, int count, double scale, int l, u64 id0, u64* out,
                   int out_cap, const u64* d_ids) {
  const int N = c->N;
  Tmp work(c, sizeof(double2) * count * (N / 2));
  Tmp ints(c, sizeof(i64) * count * N);
  encode_batch(c, z, count, scale, ints.as<i64>(), work.as<double2>());
  encrypt_coeffs(c, ints.as<i64>(), count, l, id0, out, out_cap, d_ids);
}

// ---------------------------------------------------------------- transfers
void ct_import(Context* c, Ct& ct, const u64* host_coeff, int npoly, int l, double scale) {
  GWHE_REQUIRE(ct.npoly == npoly && ct.cap >= l, ST_EINVAL, "ciphertext too small");
  const size_t N = c->N;
  for (int p = 0; p < npoly; ++p)
    GWHE_CUDA(cudaMemcpyAsync(ct.poly(p), host_coeff + (size_t)p * l * N, sizeof(u64) * l * N,
                              cudaMemcpyHostToDevice, c->stream));
  RowMap rm = rows_q(npoly, l, ct.cap);
  ntt_forward(c, ct.d, rm);
  ct.l = l;
  ct.scale = scale;
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
}

void ct_export(Context* c, const Ct& ct, u64* host_coeff) {
  const size_t N = c->N;
  Tmp t(c, sizeof(u64) * ct.npoly * ct.l * N);
  for (int p = 0; p < ct.npoly; ++p)
    GWHE_CUDA(cudaMemcpyAsync(t.u() + (size_t)p * ct.l * N, ct.poly(p), sizeof(u64) * ct.l * N,
                              cudaMemcpyDefault, c->stream));  // device or host tier
  ntt_inverse(c, t.u(), rows_q(ct.npoly, ct.l, ct.l));
  GWHE_CUDA(cudaMemcpyAsync(host_coeff, t.p, sizeof(u64) * ct.npoly * ct.l * N,
                            cudaMemcpyDeviceToHost, c->stream));
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
}

void decrypt_coeff(Context* c, const Ct& ct, u64* dev_out) {
  GWHE_REQUIRE(c->d_sk, ST_ENOKEY, "no secret key");
  decrypt_ntt(c, cpv(ct), ct.l, dev_out);
  ntt_inverse(c, dev_out, rows_q(1, ct.l, ct.l));
}

}  // namespace gwhe
