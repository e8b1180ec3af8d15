// gwas.cu -- the encrypted semi-parallel GWAS (paper section "Semi-Parallel
// GWAS with Homomorphic Encryption", Algorithms 1-11) as sequences of
// evaluator operations.
//
// Slot layouts (M = N/2 slots, nb = padded column length, B = M / nb):
//   vector v (length n)   slots 0..n-1, zeros elsewhere
//   CP matrix             one ciphertext per column (Alg. 2)
//   REP row               entry c repeated nb times: slots c*nb .. c*nb+nb-1
//   CCP matrix            column c in slots c*nb .. (Alg. 4)
//   S batch (REP)         row j: slot b*nb + t = S[j, 2b] + i S[j, 2b+1]
//   S batch (CCP)         one ciphertext: slot b*nb + t = S[t, 2b] + i S[t, 2b+1]
// The op order below is the specification that the CPU oracle's circuit
// follows as well; ciphertext bits depend on it (every key switch and rescale
// rounds).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "gwas.cuh"

namespace gwhe {

namespace {

constexpr u64 kEncX = 0x100, kEncA = 0x200, kEncY = 0x300, kEncBeta0 = 0x301, kEncDupW = 0x302,
              kEncDupWZ = 0x303, kEncXtRep = 0x10000, kEncDupM = 0x20000, kEncS = 0x1000000,
              kEncSccp = 0x100000000ull;

// mask kinds for the plaintext cache
enum MaskKind {
  kMaskSlot = 1, kMaskPrefix = 2, kMaskBlock = 3, kMaskEye = 4, kMaskHeads = 5, kMaskResidue = 6
};

// batches of the factored layout processed together (bounds the temporaries:
// d products per batch at kFactLevel limbs)
// SNP batches evaluated as one set (and, for host genotypes, staged at once)
constexpr long kSnpChunk = 64;

// eq. sigma7 coefficients of x^1, x^3, x^5, x^7 (the printed c_k / 8^k)
const double kSig[4] = {-1.73496 / 8.0, 4.19407 / 512.0, -5.43402 / 32768.0,
                        2.50739 / 2097152.0};

int ilog2(long v) {
  int r = 0;
  while ((1L << r) < v) ++r;
  return r;
}

struct Eval {
  Context* c;
  const Layout& lay;

  CtPtr fresh(int l, double scale = 1.0) { return ct_new(c, 2, l, l, scale); }

  // non-owning view of a at level l (the paper's implicit mod-drop)
  CtPtr view(const Ct& a, int l) {
    GWHE_REQUIRE(l <= a.l, ST_ELEVEL, "cannot raise a level");
    CtPtr v(new Ct());
    v->ctx = c;
    v->d = a.d;
    v->npoly = a.npoly;
    v->cap = a.cap;
    v->l = l;
    v->scale = a.scale;
    v->owned = false;
    return v;
  }
  CtPtr clone_at(const Ct& a, int l) {
    CtPtr v = view(a, l);
    return ct_clone(c, *v);
  }

  std::vector<double2> slots_zero() { return std::vector<double2>(lay.M, make_double2(0, 0)); }

  CtPtr mul_mask(const Ct& v, int kind, long idx, const std::vector<double2>& z) {
    const double ql = (double)c->mod[v.l - 1];
    const u64* pt = mask_pt(c, kind, idx, v.l, ql, z);
    CtPtr out = fresh(v.l);
    op_mul_plain(c, v, pt, ql, *out);
    op_rescale(c, *out);
    return out;
  }

  std::vector<int> pow2_steps(int count, int base = 1) {
    std::vector<int> s;
    for (int i = 0; i < count; ++i) s.push_back(base << i);
    return s;
  }

  CtPtr mac_relin_rescale(const std::vector<std::pair<const Ct*, const Ct*>>& pairs) {
    const int l = pairs[0].first->l;
    CtPtr t3 = ct_new(c, 3, l, l, 1.0);
    op_tensor_mac(c, pairs, *t3);
    CtPtr out = fresh(l);
    op_relin_rescale(c, *t3, *out);
    return out;
  }
  CtPtr mult(const Ct& a, const Ct& b) {
    CtPtr out = fresh(a.l);
    op_mult(c, a, b, *out);
    return out;
  }
  CtPtr add(const Ct& a, const Ct& b) {
    CtPtr out = fresh(a.l);
    op_addsub(c, a, b, *out, false);
    return out;
  }
  CtPtr sub(const Ct& a, const Ct& b) {
    CtPtr out = fresh(a.l);
    op_addsub(c, a, b, *out, true);
    return out;
  }
  CtPtr negate(const Ct& a) {
    CtPtr out = fresh(a.l);
    op_negate(c, a, *out);
    return out;
  }

  // Period of the shared replicate ladder for m entries: the smallest power
  // of 2^kLadderGroup >= m (at most M), so that its two step lists split
  // Alg. 1's ladder at a hoisting-group boundary and use Alg. 1's keys.
  int replicate_period(int m) const {
    int P = 1 << kLadderGroup;
    while (P < m) P <<= kLadderGroup;
    return std::min(P, lay.M);
  }
  // Alg. 1 for entries 0..m-1 of every source, each source zero beyond its m
  // entries: Alg. 1's ladder sums the rotations of the masked slot by
  // 0..M-1; here the steps P, 2P, ..., M/2 run once per source on the source
  // itself (slot s then holds v_{s mod P}), a mask keeps the slots = c mod P
  // (plaintext at scale q_last, rescale), and the steps 1, ..., P/2 fill the
  // rest.  Same sum, same depth, same keys; item r * m + c of the result is
  // entry c of source r.
  CtSetPtr replicate_all(const std::vector<const Ct*>& srcs, int m) {
    const Ct& v0 = *srcs[0];
    const int l = v0.l;
    for (const Ct* v : srcs)
      GWHE_REQUIRE(v->l == l && v->scale == v0.scale, ST_ELEVEL,
                   "replicated sources must share level and scale");
    const int P = replicate_period(m);
    CtSetPtr u = gather(srcs, l);
    if (P < lay.M) set_ladder(c, *u, pow2_steps(ilog2(lay.M / P), P));
    const double ql = (double)c->mod[l - 1];
    std::vector<const u64*> pts;
    for (int cidx = 0; cidx < m; ++cidx) {
      auto z = slots_zero();
      for (int s = cidx; s < lay.M; s += P) z[s] = make_double2(1, 0);
      pts.push_back(mask_pt(c, kMaskResidue, ((long)P << 20) | cidx, l, ql, z));
    }
    std::vector<MaskItem> mi;
    for (size_t r = 0; r < srcs.size(); ++r)
      for (int cidx = 0; cidx < m; ++cidx) mi.push_back(MaskItem{u->item((int)r), u->cap, pts[cidx]});
    CtSetPtr set = set_new(c, (int)mi.size(), 2, l, l, 1.0);
    set_mask(c, mi, u->scale, ql, *set, true);
    if (P > 1) set_ladder(c, *set, pow2_steps(ilog2(P)));
    return set;
  }
  // Alg. 2: sum_c A(c) * Replicate(v)(c), v zero beyond its m entries (as
  // every vector the circuit multiplies this way is)
  CtPtr cp_matvec(const std::vector<CtPtr>& cols, const Ct& v, int m) {
    CtSetPtr reps = replicate_all({&v}, m);
    const int lv = reps->l;
    std::vector<CtPtr> views, rv;
    std::vector<std::pair<const Ct*, const Ct*>> pairs;
    for (int cidx = 0; cidx < m; ++cidx) {
      views.push_back(view(*cols[cidx], lv));
      rv.push_back(reps->view(cidx));
      pairs.push_back({views.back().get(), rv.back().get()});
    }
    return mac_relin_rescale(pairs);
  }
  // Alg. 3 (CP-MatMult): column r of X * A is CP-MatVecMult(X, A_r); all d x m
  // replicates and the d tensor sums run as sets.
  CtSetPtr cp_matmul(const std::vector<CtPtr>& X, const std::vector<CtPtr>& Acols, int m) {
    const int d = (int)Acols.size();
    std::vector<const Ct*> srcs;
    for (int r = 0; r < d; ++r) srcs.push_back(Acols[r].get());
    CtSetPtr reps = replicate_all(srcs, m);
    const int lv = reps->l;
    std::vector<CtPtr> views, rv;
    for (int cidx = 0; cidx < m; ++cidx) views.push_back(view(*X[cidx], lv));
    std::vector<std::pair<const Ct*, const Ct*>> pairs;
    for (int r = 0; r < d; ++r)
      for (int cidx = 0; cidx < m; ++cidx) {
        rv.push_back(reps->view(r * m + cidx));
        pairs.push_back({views[cidx].get(), rv.back().get()});
      }
    CtSetPtr t3 = set_new(c, d, 3, lv, lv, 1.0);
    set_tensor_mac(c, pairs, m, *t3);
    CtSetPtr out = set_new(c, d, 2, lv, lv, 1.0);
    set_relin_rescale(c, *t3, *out);
    return out;
  }
  // A (R v): Alg. 2 over the DotProds of Alg. 6.  DotProd(R(c), v) (Alg. 5)
  // ends with (R v)_c in every slot, which is Replicate (Alg. 1) of entry c,
  // so Alg. 6's masks and Alg. 2's replicates cancel; v is taken two levels
  // lower, where the result of Alg. 6 then Alg. 2 would leave.
  CtPtr cp_rp_matvec(const std::vector<CtPtr>& acols, const std::vector<CtPtr>& rows, const Ct& v,
                     int m) {
    const int l = v.l - 2;
    GWHE_REQUIRE(l >= 2, ST_ELEVEL, "depth exhausted");
    CtPtr vv = view(v, l);
    std::vector<CtPtr> views;
    std::vector<std::pair<const Ct*, const Ct*>> pairs;
    for (int cidx = 0; cidx < m; ++cidx) {
      views.push_back(view(*rows[cidx], l));
      pairs.push_back({views.back().get(), vv.get()});
    }
    CtSetPtr dp = set_new(c, m, 2, l, l, 1.0);
    set_mult(c, pairs, *dp);
    set_ladder(c, *dp, pow2_steps(lay.logN - 1));
    const int lv = dp->l;
    std::vector<CtPtr> av, dv;
    std::vector<std::pair<const Ct*, const Ct*>> mac;
    for (int cidx = 0; cidx < m; ++cidx) {
      av.push_back(view(*acols[cidx], lv));
      dv.push_back(dp->view(cidx));
      mac.push_back({av.back().get(), dv.back().get()});
    }
    return mac_relin_rescale(mac);
  }
  // Alg. 4: log2(nb) rotate-and-add steps; block sums land at slots c*nb
  std::vector<int> colsum_steps() { return pow2_steps(ilog2(lay.nb)); }
  // Alg. 7: doubling ladder v += Rotate(v, nb 2^i) over the M/nb blocks
  std::vector<int> dup_steps() { return pow2_steps(ilog2(lay.B), lay.nb); }
  // a set holding copies of the given ciphertexts (same scale) at level l
  CtSetPtr gather(const std::vector<const Ct*>& src, int l) {
    CtSetPtr s = set_new(c, (int)src.size(), 2, l, l, src[0]->scale);
    for (size_t i = 0; i < src.size(); ++i) {
      GWHE_REQUIRE(src[i]->l >= l && src[i]->scale == src[0]->scale, ST_ELEVEL,
                   "gathered ciphertexts must reach the level and share the scale");
      for (int p = 0; p < 2; ++p)
        GWHE_CUDA(cudaMemcpyAsync(s->item((int)i) + (size_t)p * l * c->N, src[i]->poly(p),
                                  sizeof(u64) * l * c->N, cudaMemcpyDeviceToDevice, c->stream));
    }
    return s;
  }
  // in-block broadcast from the block heads: v += Rotate(v, -2^i), i < log2(nb)
  std::vector<int> bcast_steps() {
    std::vector<int> s;
    for (int i = 0; i < ilog2(lay.nb); ++i) s.push_back(-(1 << i));
    return s;
  }

  // eq. sigma7 at depth 3
  CtPtr sigma7(const Ct& x) {
    CtPtr x2 = mult(x, x);
    CtPtr x4 = mult(*x2, *x2);
    CtPtr b[4];
    for (int i = 0; i < 4; ++i) {
      b[i] = ct_clone(c, x);
      op_mul_const(c, *b[i], kSig[i]);
    }
    CtPtr t3 = mult(*b[1], *x2);
    CtPtr t7a = mult(*b[3], *x2);
    CtPtr b5 = view(*b[2], x4->l);
    CtPtr t5 = mult(*b5, *x4);
    CtPtr t7 = mult(*t7a, *x4);
    const int lv = t7->l;
    CtPtr b1v = view(*b[0], lv), t3v = view(*t3, lv);
    CtPtr r = add(*b1v, *t3v);
    op_addsub(c, *r, *t5, *r, false);
    op_addsub(c, *r, *t7, *r, false);
    op_add_const(c, *r, 0.5);
    return r;
  }

  CtPtr encrypt_vec(const std::vector<double2>& z, u64 id, int level, double scale) {
    Tmp dz(c, sizeof(double2) * lay.M);
    GWHE_CUDA(cudaMemcpyAsync(dz.p, z.data(), sizeof(double2) * lay.M, cudaMemcpyHostToDevice,
                              c->stream));
    CtPtr ct = fresh(level, scale);
    encrypt_slots(c, dz.as<double2>(), 1, scale, level, id, ct->d, ct->cap);
    return ct;
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

std::vector<double> to_host(Context* c, const double* p, size_t n) {
  std::vector<double> h(n);
  if (is_device_ptr(p)) {
    GWHE_CUDA(cudaMemcpyAsync(h.data(), p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    GWHE_CUDA(cudaStreamSynchronize(c->stream));
  } else {
    std::copy(p, p + n, h.begin());
  }
  return h;
}

}  // namespace

Layout make_layout(int logN, int n, int d, long k) {
  Layout L;
  L.logN = logN;
  L.n = n;
  L.d = d;
  L.k = k;
  L.M = 1 << (logN - 1);
  L.nb = 1 << ilog2(n);
  GWHE_REQUIRE(n >= 1 && L.nb <= L.M, ST_EINVAL, "a column of nb slots must fit one ciphertext");
  L.B = L.M / L.nb;
  L.tau = 2 * L.B;
  L.batches = (k + L.tau - 1) / L.tau;
  L.H = (n + L.B - 1) / L.B;
  return L;
}

// Give back (or free) the pinned block holding Dup(M_j), once the job's
// kernels are done with it.
static void release_dupm_host(Job* j) {
  if (!j->DupM_host || !j->c) return;
  cudaStreamSynchronize(j->c->stream);
  if (j->DupM_host_lent)
    j->c->pin_state_lent = false;
  else
    cudaFreeHost(j->DupM_host);
  j->DupM_host = nullptr;
  j->DupM_host_lent = false;
}

Job::~Job() {
  DupM.clear();
  release_dupm_host(this);
}

// Move Dup(M_j) to one pinned host block (the host tier) and point the job's
// Dup(M_j) handles at it; the device copies are dropped by the caller.
static void spill_dupm(Job* j) {
  Context* c = j->c;
  const int n = (int)j->DupM.size();
  const int l = j->DupM[0]->l;
  const size_t per = (size_t)2 * l * c->N;
  const size_t need = sizeof(u64) * per * n;
  if (!c->pin_state_lent) {
    // the context's block (grown if needed): pinned allocation and release
    // are slow and synchronise the device, so jobs reuse it
    if (c->pin_state_bytes < need) {
      if (c->pin_state) cudaFreeHost(c->pin_state);
      c->pin_state = nullptr;
      c->pin_state_bytes = 0;
      GWHE_CUDA(cudaHostAlloc(&c->pin_state, need, cudaHostAllocDefault));
      c->pin_state_bytes = need;
    }
    j->DupM_host = (u64*)c->pin_state;
    j->DupM_host_lent = true;
    c->pin_state_lent = true;
  } else {
    GWHE_CUDA(cudaHostAlloc((void**)&j->DupM_host, need, cudaHostAllocDefault));
  }
  for (int jj = 0; jj < n; ++jj) {
    const Ct& src = *j->DupM[jj];
    GWHE_REQUIRE(src.l == l, ST_ELEVEL, "Dup(M_j) at different levels");
    for (int p = 0; p < 2; ++p)
      GWHE_CUDA(cudaMemcpyAsync(j->DupM_host + jj * per + (size_t)p * l * c->N, src.poly(p),
                                sizeof(u64) * l * c->N, cudaMemcpyDeviceToHost, c->stream));
  }
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<CtPtr> hv;
  for (int jj = 0; jj < n; ++jj) {
    CtPtr v(new Ct());
    v->ctx = c;
    v->d = j->DupM_host + jj * per;
    v->cap = v->l = l;
    v->scale = j->DupM[jj]->scale;
    v->owned = false;
    hv.push_back(std::move(v));
  }
  j->DupM = std::move(hv);
}

// forget Dup(M_j), wherever it lives
static void drop_dupm(Job* j) {
  j->DupM.clear();
  release_dupm_host(j);
}

// ------------------------------------------------------------- state transfer
// The batch-invariant state of the SNP loop in one flat buffer (words):
//   header [kStateHeader]: magic, version, N, layout, n, d, cts
//   per ciphertext: level l, scale (IEEE bits)
//   then each ciphertext's residues, uint64[2][l][N], NTT domain
// Order: factored Dup(X_c) c < d, Dup((XA)_c) c < d; M-CCP Dup(M_j) j < n;
// then Dup(w), Dup(w z').
constexpr u64 kStateMagic = 0x6777686573746174ull;  // "gwhestat"
constexpr int kStateHeader = 7;

static std::vector<const Ct*> state_cts(const Job* j) {
  std::vector<const Ct*> v;
  if (j->factored) {
    for (auto& x : j->DupX) v.push_back(x.get());
    for (auto& x : j->DupB) v.push_back(x.get());
  } else {
    for (auto& x : j->DupM) v.push_back(x.get());
  }
  v.push_back(j->DupW.get());
  v.push_back(j->DupWZ.get());
  return v;
}

static size_t state_words_of(const Job* j, const std::vector<int>& levels) {
  size_t w = kStateHeader + 2 * levels.size();
  for (int l : levels) w += (size_t)2 * l * j->c->N;
  return w;
}

size_t job_state_words(const Job* j) {
  const auto v = state_cts(j);
  GWHE_REQUIRE(v.size() >= 2 && v.back() && v[v.size() - 2], ST_EINVAL,
               "covariate phase not done (fit first)");
  std::vector<int> lv;
  for (const Ct* c : v) {
    GWHE_REQUIRE(c != nullptr, ST_EINVAL, "covariate phase not done (fit first)");
    lv.push_back(c->l);
  }
  return state_words_of(j, lv);
}

void job_export_state(const Job* j, u64* buf, size_t words) {
  Context* c = j->c;
  const auto v = state_cts(j);
  GWHE_REQUIRE(words >= job_state_words(j), ST_EINVAL, "state buffer too small");
  std::vector<u64> head(kStateHeader + 2 * v.size());
  head[0] = kStateMagic;
  head[1] = 1;
  head[2] = (u64)c->N;
  head[3] = j->factored ? kLayoutFactored : kLayoutMccp;
  head[4] = (u64)j->lay.n;
  head[5] = (u64)j->lay.d;
  head[6] = (u64)v.size();
  for (size_t i = 0; i < v.size(); ++i) {
    head[kStateHeader + 2 * i] = (u64)v[i]->l;
    std::memcpy(&head[kStateHeader + 2 * i + 1], &v[i]->scale, sizeof(double));
  }
  GWHE_CUDA(cudaMemcpyAsync(buf, head.data(), sizeof(u64) * head.size(), cudaMemcpyDefault,
                            c->stream));
  size_t off = head.size();
  for (const Ct* ct : v)
    for (int p = 0; p < 2; ++p) {
      // Dup(M_j) may live in the pinned host tier
      GWHE_CUDA(cudaMemcpyAsync(buf + off, ct->poly(p), sizeof(u64) * ct->l * c->N,
                                cudaMemcpyDefault, c->stream));
      off += (size_t)ct->l * c->N;
    }
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
}

void job_import_state(Job* j, const u64* buf, size_t words) {
  Context* c = j->c;
  GWHE_REQUIRE(words >= (size_t)kStateHeader, ST_EINVAL, "state buffer too small");
  std::vector<u64> head(kStateHeader);
  GWHE_CUDA(cudaMemcpyAsync(head.data(), buf, sizeof(u64) * kStateHeader, cudaMemcpyDefault,
                            c->stream));
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
  const size_t cnt = head[6];
  const size_t want_cnt = j->factored ? 2 * (size_t)j->lay.d + 2 : (size_t)j->lay.n + 2;
  GWHE_REQUIRE(head[0] == kStateMagic && head[1] == 1 && head[2] == (u64)c->N &&
                   head[3] == (u64)(j->factored ? kLayoutFactored : kLayoutMccp) &&
                   head[4] == (u64)j->lay.n && head[5] == (u64)j->lay.d && cnt == want_cnt,
               ST_EINVAL, "the state buffer was made for another job shape or ring");
  j->sprime_pre.clear();
  std::vector<u64> meta(2 * cnt);
  GWHE_CUDA(cudaMemcpyAsync(meta.data(), buf + kStateHeader, sizeof(u64) * meta.size(),
                            cudaMemcpyDefault, c->stream));
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<int> lv(cnt);
  for (size_t i = 0; i < cnt; ++i) {
    lv[i] = (int)meta[2 * i];
    GWHE_REQUIRE(lv[i] >= 1 && lv[i] <= c->P.L, ST_EINVAL, "bad level in the state buffer");
  }
  GWHE_REQUIRE(words >= state_words_of(j, lv), ST_EINVAL, "state buffer too small");
  std::vector<CtPtr> cts;
  size_t off = kStateHeader + 2 * cnt;
  for (size_t i = 0; i < cnt; ++i) {
    double sc;
    std::memcpy(&sc, &meta[2 * i + 1], sizeof(double));
    CtPtr ct = ct_new(c, 2, lv[i], lv[i], sc);
    for (int p = 0; p < 2; ++p) {
      GWHE_CUDA(cudaMemcpyAsync(ct->poly(p), buf + off, sizeof(u64) * lv[i] * c->N,
                                cudaMemcpyDefault, c->stream));
      off += (size_t)lv[i] * c->N;
    }
    cts.push_back(std::move(ct));
  }
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
  drop_dupm(j);
  j->DupX.clear();
  j->DupB.clear();
  size_t it = 0;
  if (j->factored) {
    for (int cc = 0; cc < j->lay.d; ++cc) j->DupX.push_back(std::move(cts[it++]));
    for (int cc = 0; cc < j->lay.d; ++cc) j->DupB.push_back(std::move(cts[it++]));
  } else {
    for (int jj = 0; jj < j->lay.n; ++jj) j->DupM.push_back(std::move(cts[it++]));
    if (j->dupm_chunk > 0) spill_dupm(j);
  }
  j->DupW = std::move(cts[it++]);
  j->DupWZ = std::move(cts[it++]);
}

void job_set_host_state(Job* j, int chunk) {
  GWHE_REQUIRE(chunk >= 0, ST_EINVAL, "negative chunk");
  GWHE_REQUIRE(!j->DupM_host || chunk > 0, ST_EINVAL, "Dup(M_j) already in host memory");
  j->dupm_chunk = chunk;
}

Job* job_create(Context* c, int n, int d, long k, int mode) {
  GWHE_REQUIRE(d >= 1 && d <= 64 && k >= 1, ST_EINVAL, "bad job shape");
  GWHE_REQUIRE(mode == kLayoutAuto || mode == kLayoutMccp || mode == kLayoutFactored, ST_EINVAL,
               "bad layout mode");
  Job* j = new Job();
  j->c = c;
  j->lay = make_layout(c->logN, n, d, k);
  // auto: the factored layout whenever the ring can run the fit (it is the
  // faster one at every cohort size measured and the only one past n = 256);
  // M-CCP on rings without the fit's depth (split mode)
  j->factored = mode == kLayoutFactored || (mode == kLayoutAuto && c->P.L > kMLevel);
  return j;
}

void job_set_nonce(Job* j, u32 nonce) {
  GWHE_REQUIRE(nonce <= kMaxNonce, ST_EINVAL, "job nonce out of range");
  GWHE_REQUIRE(j->X.empty() && !j->y, ST_EINVAL, "set the nonce before encrypting the inputs");
  j->enc_base = (u64)nonce << kNonceShift;
}

void job_release_results(Job* j) {
  // the kept outputs are views into sets the job owns: drop both (the
  // covariate state's sets stay)
  for (auto& o : j->out)
    for (auto& v : o) v.reset();
  j->out.clear();
  auto& sets = j->sets;
  sets.erase(std::remove_if(sets.begin(), sets.end(),
                            [&](const CtSetPtr& s) { return s->is_output; }),
             sets.end());
}

std::vector<int> job_rotation_steps(const Job* j) {
  // every rotation of the circuit's ladders (Replicate and DotProd over all
  // slots, colSum over nb, Duplicate over the blocks, the factored layout's
  // in-block broadcast), as the hoisted groups evaluate them
  const Layout& lay = j->lay;
  std::vector<std::vector<int>> ladders(4);
  for (int i = 0; i < lay.logN - 1; ++i) ladders[0].push_back(1 << i);
  for (int i = 0; i < ilog2(lay.nb); ++i) ladders[1].push_back(1 << i);
  for (int i = 0; i < ilog2(lay.B); ++i) ladders[2].push_back(lay.nb << i);
  if (j->factored)
    for (int i = 0; i < ilog2(lay.nb); ++i) ladders[3].push_back(-(1 << i));
  std::vector<int> s;
  for (const auto& steps : ladders)
    for (const auto& g : ladder_groups(steps))
      for (int r : g)
        if (std::find(s.begin(), s.end(), r) == s.end()) s.push_back(r);
  return s;
}

// The Alg. 9 / Alg. 11 inputs at the top level, encryption ids as in the
// spec: with kInCov X (CP), (X^T X)^-1 (CP) and, in the M-CCP layout, X^T as
// REP; with kInPheno y and beta0 = Enc(0).  All requested ciphertexts are
// encoded and encrypted as one batch.
enum { kInCov = 1, kInPheno = 2 };
static void encrypt_input_parts(Job* j, const double* Xp, const double* Ap, const double* yp,
                                int parts) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  const int n = lay.n, d = lay.d, L = c->P.L, M = lay.M;
  const double delta = std::ldexp(1.0, c->P.scale_bits);
  const bool cov = parts & kInCov, pheno = parts & kInPheno;
  if (cov) j->sprime_pre.clear();  // S' made from the previous covariates
  std::vector<double> X, A, y;
  if (cov) {
    X = to_host(c, Xp, (size_t)n * d);
    A = to_host(c, Ap, (size_t)d * d);
  }
  if (pheno) y = to_host(c, yp, n);
  // the factored layout has no CCP matrix M and needs no X^T
  const int H = j->factored ? 0 : lay.H;
  const int cnt = (cov ? 2 * d + d * H : 0) + (pheno ? 2 : 0);
  std::vector<double2> z((size_t)cnt * M, make_double2(0, 0));
  std::vector<u64> ids(cnt);
  int it = 0;
  if (cov) {
    for (int col = 0; col < d; ++col, ++it) {
      ids[it] = j->enc_base + kEncX + col;
      for (int t = 0; t < n; ++t) z[(size_t)it * M + t] = make_double2(X[(size_t)t * d + col], 0);
    }
    for (int col = 0; col < d; ++col, ++it) {
      ids[it] = j->enc_base + kEncA + col;
      for (int r = 0; r < d; ++r) z[(size_t)it * M + r] = make_double2(A[(size_t)r * d + col], 0);
    }
  }
  if (pheno) {
    ids[it] = j->enc_base + kEncY;
    for (int t = 0; t < n; ++t) z[(size_t)it * M + t] = make_double2(y[t], 0);
    ++it;
    ids[it++] = j->enc_base + kEncBeta0;
  }
  if (cov)
    for (int col = 0; col < d; ++col)
      for (int h = 0; h < H; ++h, ++it) {
        ids[it] = j->enc_base + kEncXtRep + (u64)col * 4096 + h;
        for (int b = 0; b < lay.B; ++b) {
          const int s = h * lay.B + b;
          if (s >= n) continue;
          for (int t = 0; t < lay.nb; ++t)
            z[(size_t)it * M + b * lay.nb + t] = make_double2(X[(size_t)s * d + col], 0);
        }
      }
  CtSetPtr in = set_new(c, cnt, 2, L, L, delta);
  {
    Tmp dz(c, sizeof(double2) * z.size()), did(c, sizeof(u64) * cnt);
    GWHE_CUDA(cudaMemcpyAsync(dz.p, z.data(), sizeof(double2) * z.size(), cudaMemcpyHostToDevice,
                              c->stream));
    GWHE_CUDA(cudaMemcpyAsync(did.p, ids.data(), sizeof(u64) * cnt, cudaMemcpyHostToDevice,
                              c->stream));
    encrypt_slots(c, dz.as<double2>(), cnt, delta, L, 0, in->d, L, did.u());
  }
  it = 0;
  if (cov) {
    j->X.clear();
    j->A.clear();
    j->XtREP.clear();
    j->XtREP.resize(d);
    for (int col = 0; col < d; ++col) j->X.push_back(in->view(it++));
    for (int col = 0; col < d; ++col) j->A.push_back(in->view(it++));
  }
  if (pheno) {
    j->y = in->view(it++);
    j->beta0 = in->view(it++);
  }
  if (cov)
    for (int col = 0; col < d; ++col)
      for (int h = 0; h < H; ++h) j->XtREP[col].push_back(in->view(it++));
  j->sets.push_back(std::move(in));
}

void job_encrypt_inputs(Job* j, const double* Xp, const double* Ap, const double* yp) {
  encrypt_input_parts(j, Xp, Ap, yp, kInCov | kInPheno);
}
void job_encrypt_covariates(Job* j, const double* Xp, const double* Ap) {
  encrypt_input_parts(j, Xp, Ap, nullptr, kInCov);
}
void job_encrypt_phenotype(Job* j, const double* yp) {
  encrypt_input_parts(j, nullptr, nullptr, yp, kInPheno);
}

static void make_dup_state(Job* j, Eval& ev) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  const int lb = kBatchLevel;
  GWHE_REQUIRE(j->wzp->l >= lb - 1, ST_ELEVEL, "depth exhausted before the SNP batches");
  drop_dupm(j);
  if (!j->factored) {
  // Dup(M_j) for every column j: mask block (j mod B) of ciphertext j / B at
  // lb + 1 limbs (plaintext at scale q_last, rescale), then Alg. 7's ladder
  std::vector<CtPtr> src;
  for (auto& m : j->Mct) src.push_back(ev.view(*m, lb + 1));
  const double ql = (double)c->mod[lb];
  std::vector<MaskItem> mi;
  for (int jj = 0; jj < lay.n; ++jj) {
    const int h = jj / lay.B, b = jj % lay.B;
    auto z = ev.slots_zero();
    for (int t = 0; t < lay.n; ++t) z[b * lay.nb + t] = make_double2(1, 0);
    const long key = ((long)lay.n << 32) | ((long)lay.nb << 16) | b;
    mi.push_back(MaskItem{src[h]->d, src[h]->cap, mask_pt(c, kMaskBlock, key, lb + 1, ql, z)});
  }
  CtSetPtr dm = set_new(c, lay.n, 2, lb + 1, lb + 1, 1.0);
  set_mask(c, mi, src[0]->scale, ql, *dm, true);
  set_ladder(c, *dm, ev.dup_steps());
  for (int jj = 0; jj < lay.n; ++jj) j->DupM.push_back(dm->view(jj));
  if (j->dupm_chunk > 0)
    spill_dupm(j);  // dm (the device copy) is freed at scope exit
  else
    j->sets.push_back(std::move(dm));
  }
  // Dup(w) and Dup(w z') (Alg. 7) share one ladder set: the ladder's key
  // switches and sums do not read the scales, so each view keeps its source's
  CtSetPtr dd = set_new(c, 2, 2, lb - 1, lb - 1, 1.0);
  const Ct* dsrc[2] = {j->w_m.get(), j->wzp.get()};
  for (int i = 0; i < 2; ++i) {
    GWHE_REQUIRE(dsrc[i]->l >= lb - 1, ST_ELEVEL, "depth exhausted before the SNP batches");
    for (int p = 0; p < 2; ++p)
      GWHE_CUDA(cudaMemcpyAsync(dd->item(i) + (size_t)p * (lb - 1) * c->N, dsrc[i]->poly(p),
                                sizeof(u64) * (lb - 1) * c->N, cudaMemcpyDeviceToDevice,
                                c->stream));
  }
  set_ladder(c, *dd, ev.dup_steps());
  j->DupW = dd->view(0);
  j->DupW->scale = j->w_m->scale;
  j->DupWZ = dd->view(1);
  j->DupWZ->scale = j->wzp->scale;
  j->sets.push_back(std::move(dd));
}

// An independent chain of operations on a second stream of the job's
// context: fork() orders the side stream after the work queued so far and
// makes the context issue there, leave() returns to the main stream, and
// join() makes the main stream wait for everything the chain issued.  Both
// streams share the context's memory pool (stream-ordered: the fork and
// join events order reuse across them) and its mask cache (a mask encoded on
// one stream is waited for on the other).  The side stream has the main
// stream's priority, or with raise = true the next higher one (for the
// critical chain when other work fills the GPU beside it).  With the
// kernel-class timers on, the chain stays on the main stream: the timers'
// per-class times would otherwise count the overlap twice.
struct SideChain {
  Context* c;
  cudaStream_t main, side = nullptr;
  cudaEvent_t ev = nullptr;
  bool on_side = false, joined = true;
  explicit SideChain(Context* c_, bool raise = false) : c(c_), main(c_->stream) {
    if (c->prof.on) return;
    int prio = 0;
    if (cudaStreamGetPriority(main, &prio) != cudaSuccess) {
      cudaGetLastError();
      prio = 0;
    }
    if (raise) {
      int least = 0, greatest = 0;
      GWHE_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      prio = std::max(greatest, prio - 1);  // numerically lower = higher priority
    }
    GWHE_CUDA(cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio));
    GWHE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  void fork() {
    if (!side) return;
    GWHE_CUDA(cudaEventRecord(ev, main));
    GWHE_CUDA(cudaStreamWaitEvent(side, ev, 0));
    c->stream = side;
    on_side = true;
    joined = false;
  }
  void leave() {
    c->stream = main;
    on_side = false;
  }
  void join() {
    if (!side) return;
    GWHE_CUDA(cudaEventRecord(ev, side));
    GWHE_CUDA(cudaStreamWaitEvent(main, ev, 0));
    joined = true;
  }
  ~SideChain() {
    c->stream = main;
    if (!side) return;
    if (!joined && cudaEventRecord(ev, side) == cudaSuccess) cudaStreamWaitEvent(main, ev, 0);
    cudaStreamDestroy(side);  // released once its work is done
    cudaEventDestroy(ev);
  }
};

namespace {
void precompute_sprime(Job* j, Eval& ev);
}  // namespace

void job_fit(Job* j, int kappa) {
  GWHE_REQUIRE(kappa >= 1, ST_EINVAL, "kappa >= 1");
  GWHE_REQUIRE(!j->X.empty() && j->y && j->beta0, ST_EINVAL,
               "inputs not encrypted (covariates and phenotype)");
  Context* c = j->c;
  const Layout& lay = j->lay;
  Eval ev{c, lay};
  const int d = lay.d, n = lay.n;
  // X A: Alg. 3 (CP-MatMult) from X and A dropped to kMLevel limbs, every
  // column duplicated into all blocks (Alg. 7), and in the factored layout
  // Dup(X_c) at kFactLevel: they read only the encrypted inputs, so they run
  // on a second stream beside Alg. 9 and eqs. z, zprime
  if (j->factored)
    GWHE_REQUIRE(j->X[0]->l >= kFactLevel, ST_ELEVEL, "need kFactLevel limbs for Dup(X_c)");
  // factored layout with SNP batches already encrypted: their S' (eq. Sprime,
  // second form) needs only Dup(X_c) and Dup((XA)_c), so the second stream
  // goes on from those to the batches' S' while the fit's chain, the critical
  // path, runs on a stream of higher priority
  const bool pre = j->factored && !j->enc_snps.empty();
  j->sprime_pre.clear();
  SideChain side(c);
  side.fork();
  std::vector<CtPtr> Alow;
  for (int rr = 0; rr < d; ++rr) Alow.push_back(ev.view(*j->A[rr], kMLevel));
  CtSetPtr xa = ev.cp_matmul(j->X, Alow, d);
  set_ladder(c, *xa, ev.dup_steps());  // Duplicate(XA_r) for every r
  CtSetPtr dx;
  if (j->factored) {
    std::vector<const Ct*> xs;
    for (int cc = 0; cc < d; ++cc) xs.push_back(j->X[cc].get());
    dx = ev.gather(xs, kFactLevel);
    set_ladder(c, *dx, ev.dup_steps());
  }
  if (pre) {
    j->DupB.clear();
    j->DupX.clear();
    for (int rr = 0; rr < d; ++rr) j->DupB.push_back(xa->view(rr));
    for (int cc = 0; cc < d; ++cc) j->DupX.push_back(dx->view(cc));
    precompute_sprime(j, ev);
  }
  side.leave();
  SideChain fit(c, true);
  if (pre) fit.fork();
  // Alg. 9
  CtPtr beta = ev.clone_at(*j->beta0, j->beta0->l);
  CtPtr p, ymp;
  for (int it = 0; it < kappa; ++it) {
    CtPtr xb = ev.cp_matvec(j->X, *beta, d);
    p = ev.sigma7(*xb);
    CtPtr yv = ev.view(*j->y, p->l);
    ymp = ev.sub(*yv, *p);
    CtPtr ag = ev.cp_rp_matvec(j->A, j->X, *ymp, d);  // A g, g = X^T (y - p)
    op_mul_int(c, *ag, 4);
    CtPtr bv = ev.view(*beta, ag->l);
    beta = ev.sub(*bv, *ag);
  }
  j->beta = ev.clone_at(*beta, beta->l);
  // X beta of eq. z (Alg. 2) needs only beta: on its own stream beside the
  // weights and Alg. 10
  SideChain side_xb(c);
  side_xb.fork();
  CtPtr xb = ev.cp_matvec(j->X, *beta, d);
  side_xb.leave();
  // w = p (1 - p); the masked copy feeds Dup(w) and w z'
  CtPtr omp = ev.negate(*p);
  op_add_const(c, *omp, 1.0);
  CtPtr w = ev.mult(*p, *omp);
  {
    auto z = ev.slots_zero();
    for (int t = 0; t < n; ++t) z[t] = make_double2(1, 0);
    j->w_m = ev.mul_mask(*w, kMaskPrefix, ((long)n << 16) | lay.nb, z);
  }
  // Alg. 10: guess 3; the first step multiplies by integers only
  CtPtr g = ct_clone(c, *w);
  op_mul_int(c, *g, 3);
  {
    CtPtr u = ev.negate(*g);
    op_add_const(c, *u, 2.0);
    op_mul_int(c, *u, 3);
    g = std::move(u);
  }
  for (int it = 0; it < 2; ++it) {
    CtPtr wv = ev.view(*w, g->l);
    CtPtr t = ev.mult(*wv, *g);
    CtPtr u = ev.negate(*t);
    op_add_const(c, *u, 2.0);
    CtPtr gv = ev.view(*g, u->l);
    g = ev.mult(*gv, *u);
  }
  CtPtr winv = std::move(g);
  // eq. z
  int lv = std::min(winv->l, ymp->l);
  CtPtr wi = ev.view(*winv, lv), ym = ev.view(*ymp, lv);
  CtPtr r = ev.mult(*wi, *ym);
  side_xb.join();
  lv = std::min(xb->l, r->l);
  CtPtr xbv = ev.view(*xb, lv), rv = ev.view(*r, lv);
  j->z = ev.add(*xbv, *rv);
  // eq. zprime, second form: z' = z - X (A (X^T z))
  CtPtr axtz = ev.cp_rp_matvec(j->A, j->X, *j->z, d);
  CtPtr xaxtz = ev.cp_matvec(j->X, *axtz, d);
  CtPtr zv = ev.view(*j->z, xaxtz->l);
  j->zp = ev.sub(*zv, *xaxtz);
  CtPtr wmv = ev.view(*j->w_m, j->zp->l);
  j->wzp = ev.mult(*wmv, *j->zp);
  if (pre) {
    make_dup_state(j, ev);
    fit.leave();
    fit.join();
  }
  side.join();
  if (j->factored) {
    // second form of eq. Sprime: keep Dup((XA)_c) and Dup(X_c) at kFactLevel
    j->DupB.clear();
    j->DupX.clear();
    for (int rr = 0; rr < d; ++rr) j->DupB.push_back(xa->view(rr));
    j->sets.push_back(std::move(xa));
    for (int cc = 0; cc < d; ++cc) j->DupX.push_back(dx->view(cc));
    j->sets.push_back(std::move(dx));
    if (!pre) make_dup_state(j, ev);
    return;
  }
  // eq. M = I - X A X^T: Alg. 8 (CP-REP-MatMult) on the duplicated columns
  const int l0 = xa->l;
  std::vector<CtPtr> dv, xv;
  for (int rr = 0; rr < d; ++rr) dv.push_back(xa->view(rr));
  std::vector<std::pair<const Ct*, const Ct*>> pairs;
  for (int h = 0; h < lay.H; ++h)
    for (int rr = 0; rr < d; ++rr) {
      xv.push_back(ev.view(*j->XtREP[rr][h], l0));
      pairs.push_back({dv[rr].get(), xv.back().get()});
    }
  CtSetPtr t3 = set_new(c, lay.H, 3, l0, l0, 1.0);
  set_tensor_mac(c, pairs, d, *t3);
  CtSetPtr acc = set_new(c, lay.H, 2, l0, l0, 1.0);
  set_relin_rescale(c, *t3, *acc);
  j->Mct.clear();
  for (int h = 0; h < lay.H; ++h) {
    CtPtr ah = acc->view(h);
    CtPtr m = ev.negate(*ah);
    auto z = ev.slots_zero();
    for (int b = 0; b < lay.B; ++b) {
      const int col = h * lay.B + b;
      if (col < n) z[b * lay.nb + col] = make_double2(1, 0);
    }
    const u64* pt = mask_pt(c, kMaskEye, ((long)n << 32) | ((long)lay.nb << 16) | h, m->l,
                            m->scale, z);
    op_add_plain(c, *m, pt);
    j->Mct.push_back(std::move(m));
  }
  make_dup_state(j, ev);
}

void job_set_fit_state(Job* j, const double* Mp, const double* wp, const double* wzp) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  Eval ev{c, lay};
  const int n = lay.n, lb = kBatchLevel;
  GWHE_REQUIRE(!j->factored, ST_EINVAL, "split mode needs the M-CCP layout");
  GWHE_REQUIRE(c->P.L >= lb, ST_ELEVEL, "need at least 4 limbs for the SNP batches");
  const double delta = std::ldexp(1.0, c->P.scale_bits);
  const std::vector<double> M = to_host(c, Mp, (size_t)n * n), w = to_host(c, wp, n),
                            wz = to_host(c, wzp, n);
  auto dup = [&](const std::vector<double>& v, size_t stride, size_t off) {
    auto z = ev.slots_zero();
    for (int b = 0; b < lay.B; ++b)
      for (int t = 0; t < n; ++t) z[b * lay.nb + t] = make_double2(v[(size_t)t * stride + off], 0);
    return z;
  };
  drop_dupm(j);
  for (int jj = 0; jj < n; ++jj)
    j->DupM.push_back(ev.encrypt_vec(dup(M, n, jj), j->enc_base + kEncDupM + jj, lb, delta));
  if (j->dupm_chunk > 0) spill_dupm(j);
  j->DupW = ev.encrypt_vec(dup(w, 1, 0), j->enc_base + kEncDupW, lb - 1, delta);
  j->DupWZ = ev.encrypt_vec(dup(wz, 1, 0), j->enc_base + kEncDupWZ, lb - 1, delta);
}

namespace {

// the Alg. 11 loop body after S' (at kBatchLevel - 1 limbs) for batches
// [b0, b0 + nbt): numerator = colSum(Dup(w z') S'), WS' = Dup(w) S',
// WSS = WS' S', WSC = WS' conj(S'), denEven/denOdd (the 1/2 as scale
// metadata), colSum of each; the outputs become the job's kept results
void batch_body(Job* j, Eval& ev, CtSetPtr Sp, long b0) {
  Context* c = j->c;
  const int lb = kBatchLevel, nbt = Sp->cnt;
  std::vector<CtPtr> spv;
  for (int i = 0; i < nbt; ++i) spv.push_back(Sp->view(i));
  // numerator = colSum(Dup(w z') S'): its own chain on a second stream,
  // beside the denominators' (both only read S'); their launches at 1-3
  // limbs fill the GPU together
  SideChain side(c);
  side.fork();
  CtSetPtr num = set_new(c, nbt, 2, lb - 1, lb - 1, 1.0);
  {
    std::vector<std::pair<const Ct*, const Ct*>> pr;
    for (int i = 0; i < nbt; ++i) pr.push_back({j->DupWZ.get(), spv[i].get()});
    set_mult(c, pr, *num);
  }
  set_ladder(c, *num, ev.colsum_steps());
  side.leave();
  // WS' = Dup(w) S'
  CtSetPtr ws = set_new(c, nbt, 2, lb - 1, lb - 1, 1.0);
  {
    std::vector<std::pair<const Ct*, const Ct*>> pr;
    for (int i = 0; i < nbt; ++i) pr.push_back({j->DupW.get(), spv[i].get()});
    set_mult(c, pr, *ws);
  }
  // conj(S') at lb - 2; WSS = WS' S', WSC = WS' conj(S') as one set of 2 nbt
  CtSet s1 = Sp->slice(0, nbt, lb - 2);
  CtSetPtr cj = set_new(c, nbt, 2, lb - 2, lb - 2, 1.0);
  set_galois(c, s1, galois_conj(c), *cj);
  CtSetPtr W2 = set_new(c, 2 * nbt, 2, lb - 2, lb - 2, 1.0);
  {
    std::vector<CtPtr> keep;
    std::vector<std::pair<const Ct*, const Ct*>> pr;
    for (int i = 0; i < nbt; ++i) {
      keep.push_back(ws->view(i));
      keep.push_back(s1.view(i));
      pr.push_back({keep[keep.size() - 2].get(), keep.back().get()});
    }
    for (int i = 0; i < nbt; ++i) {
      keep.push_back(ws->view(i));
      keep.push_back(cj->view(i));
      pr.push_back({keep[keep.size() - 2].get(), keep.back().get()});
    }
    set_mult(c, pr, *W2);
  }
  // denEven = WSC + WSS, denOdd = WSC - WSS (the 1/2 as scale metadata), colSum
  CtSetPtr D = set_new(c, 2 * nbt, 2, lb - 3, lb - 3, 1.0);
  {
    const int l = W2->l;
    Ct wss = W2->slice(0, nbt, l).all(), wsc = W2->slice(nbt, nbt, l).all();
    Ct de = D->slice(0, nbt, l).all(), dO = D->slice(nbt, nbt, l).all();
    op_addsub(c, wsc, wss, de, false);
    op_addsub(c, wsc, wss, dO, true);
    D->l = l;
    D->scale = W2->scale * 2.0;
  }
  set_ladder(c, *D, ev.colsum_steps());
  side.join();
  for (int i = 0; i < nbt; ++i)
    j->out[b0 + i] = {num->view(i), D->view(i), D->view(nbt + i)};
  num->is_output = true;
  D->is_output = true;
  j->sets.push_back(std::move(num));
  j->sets.push_back(std::move(D));
}

// Host-to-device copies into two device slots on a copy stream, for
// prefetching the next chunk while the compute stream works on the current
// one.  copy(s, ...) queues the copy once the compute stream has released
// slot s (release(s) after the work that reads it) and makes the compute
// stream wait for the copy; wait_copied(s) blocks the host until the slot's
// last copy has left its source.  Waits are on CUDA events, which complete or
// fail.
struct TwoSlotCopy {
  Context* c;
  size_t cap;
  std::unique_ptr<Tmp> dev[2];
  cudaStream_t cs = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  TwoSlotCopy(Context* c_, size_t cap_bytes) : c(c_), cap(cap_bytes) {
    try {
      GWHE_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      for (int s = 0; s < 2; ++s) {
        dev[s].reset(new Tmp(c, cap));
        GWHE_CUDA(cudaEventCreateWithFlags(&copied[s], cudaEventDisableTiming));
        GWHE_CUDA(cudaEventCreateWithFlags(&freed[s], cudaEventDisableTiming));
      }
      // the slots come from the compute stream's pool
      GWHE_CUDA(cudaEventRecord(freed[0], c->stream));
      GWHE_CUDA(cudaStreamWaitEvent(cs, freed[0], 0));
    } catch (...) {
      destroy();
      throw;
    }
  }
  void wait_copied(int s) {
    if (used[s]) GWHE_CUDA(cudaEventSynchronize(copied[s]));
  }
  void* copy(int s, const void* src, size_t bytes) {
    GWHE_REQUIRE(bytes >= 1 && bytes <= cap, ST_EINVAL, "staged chunk too large");
    if (used[s]) GWHE_CUDA(cudaStreamWaitEvent(cs, freed[s], 0));
    GWHE_CUDA(cudaMemcpyAsync(dev[s]->p, src, bytes, cudaMemcpyHostToDevice, cs));
    GWHE_CUDA(cudaEventRecord(copied[s], cs));
    GWHE_CUDA(cudaStreamWaitEvent(c->stream, copied[s], 0));
    used[s] = true;
    return dev[s]->p;
  }
  void release(int s) { GWHE_CUDA(cudaEventRecord(freed[s], c->stream)); }
  void destroy() {
    if (cs) cudaStreamSynchronize(cs);
    for (int s = 0; s < 2; ++s) {
      if (copied[s]) cudaEventDestroy(copied[s]);
      if (freed[s]) cudaEventDestroy(freed[s]);
      copied[s] = freed[s] = nullptr;
    }
    if (cs) cudaStreamDestroy(cs);
    cs = nullptr;
  }
  ~TwoSlotCopy() {
    // the copy stream is drained; the slots then go back to the compute
    // stream's pool in stream order, after the work queued there that reads
    // them (the compute stream waited for every copy), with no host wait
    destroy();
  }
};

// Genotype column ranges from host memory: stage() gathers the n row
// segments [col0, col0 + w) into the slot's pinned buffer (after the slot's
// previous copy has left it) and copies them to the device.  The pinned
// buffers belong to the context and are reused by later calls.
struct HostStager {
  int n;
  long wmax;
  double* pin[2] = {nullptr, nullptr};
  TwoSlotCopy cp;
  HostStager(Context* c, int n_, long wmax_)
      : n(n_), wmax(wmax_), cp(c, sizeof(double) * (size_t)n_ * wmax_) {
    // any job's set of 64 batches fits n x 64 tau <= 64 N doubles (n <= nb,
    // tau = N / nb): the buffers are allocated at that size once per context,
    // since pinned allocation and release synchronise the whole device
    const size_t need = std::max(sizeof(double) * (size_t)n * wmax,
                                 sizeof(double) * (size_t)kSnpChunk * c->N);
    if (c->pin_stage_bytes < need) {
      for (void*& p : c->pin_stage) {
        if (p) cudaFreeHost(p);
        p = nullptr;
      }
      c->pin_stage_bytes = 0;
      for (void*& p : c->pin_stage)
        if (cudaHostAlloc(&p, need, cudaHostAllocDefault) != cudaSuccess) {
          cudaGetLastError();
          p = nullptr;
          throw Error(ST_ENOMEM, "pinned staging allocation failed");
        }
      c->pin_stage_bytes = need;
    }
    for (int s = 0; s < 2; ++s) pin[s] = (double*)c->pin_stage[s];
  }
  const double* stage(int s, const double* S, long k, long col0, long w) {
    GWHE_REQUIRE(w >= 1 && w <= wmax, ST_EINVAL, "staged column range too wide");
    cp.wait_copied(s);
    for (int t = 0; t < n; ++t)
      std::memcpy(pin[s] + (size_t)t * w, S + (size_t)t * k + col0, sizeof(double) * w);
    return (const double*)cp.copy(s, pin[s], sizeof(double) * (size_t)n * w);
  }
  void release(int s) { cp.release(s); }
  ~HostStager() {
    // the context's buffers must be free for the next call
    cp.wait_copied(0);
    cp.wait_copied(1);
  }
};

// genotype columns col0.. of every sample on the device, row pitch ld
struct SnpSrc {
  const double* S;
  long ld, col0;
};

// M-CCP layout: per batch encode + encrypt the n REP rows, then the tensor
// sum of Alg. 8 (S' = sum_j Dup(M_j) S_ij), relinearise and rescale
CtSetPtr sprime_mccp(Job* j, const SnpSrc* src, long b0, long b1) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  const int n = lay.n, lb = kBatchLevel, N = c->N;
  const double delta = std::ldexp(1.0, c->P.scale_bits);
  const int nbt = (int)(b1 - b0);
  CtSetPtr T3 = set_new(c, nbt, 3, lb, lb, 1.0);
  // Dup(M_j) for columns [j0, j0 + J) at a time: on the device, one chunk of
  // all n; in the host tier, chunks prefetched into two device slots, each
  // used by every batch of the set (the partial tensor sums accumulate)
  const bool host = j->DupM_host != nullptr;
  const int J = host ? std::min(n, j->dupm_chunk) : n;
  const size_t per = (size_t)2 * lb * N;
  std::unique_ptr<TwoSlotCopy> cp;
  if (host) {
    GWHE_REQUIRE(j->DupM[0]->l == lb, ST_ELEVEL, "Dup(M_j) not at the batch level");
    cp.reset(new TwoSlotCopy(c, sizeof(u64) * per * J));
  }
  // the rows are encrypted here from the genotypes (src) or were encrypted
  // ahead of the loop (job_encrypt_snps)
  Tmp z(c, src ? sizeof(double2) * (size_t)J * lay.M : 8);
  Tmp sct(c, src ? sizeof(u64) * (size_t)J * per : 8);
  std::vector<Ct> srow(J), dm(J);
  for (int jj = 0; jj < J; ++jj) {
    srow[jj].ctx = dm[jj].ctx = c;
    srow[jj].d = sct.u() + (size_t)jj * per;
    srow[jj].cap = srow[jj].l = dm[jj].cap = dm[jj].l = lb;
    srow[jj].scale = delta;
    srow[jj].owned = dm[jj].owned = false;
  }
  for (int j0 = 0, ci = 0; j0 < n; j0 += J, ++ci) {
    const int jn = std::min(J, n - j0);
    std::vector<std::pair<const Ct*, const Ct*>> pairs;
    if (host) {
      const u64* dd = (const u64*)cp->copy(ci & 1, j->DupM_host + (size_t)j0 * per,
                                           sizeof(u64) * per * jn);
      for (int jj = 0; jj < jn; ++jj) {
        dm[jj].d = (u64*)dd + (size_t)jj * per;
        dm[jj].scale = j->DupM[j0 + jj]->scale;
        pairs.push_back({&dm[jj], &srow[jj]});
      }
    } else {
      for (int jj = 0; jj < jn; ++jj) pairs.push_back({j->DupM[j0 + jj].get(), &srow[jj]});
    }
    for (long bi = b0; bi < b1; ++bi) {
      std::vector<CtPtr> rows;
      if (src) {
        // REP rows j0 .. j0 + jn of batch bi (encryption ids per sample row)
        build_snp_rep(c, src->S + (size_t)j0 * src->ld, src->ld, src->col0, jn, lay.k,
                      bi * lay.tau, lay.nb, lay.B, lay.M, z.as<double2>());
        encrypt_slots(c, z.as<double2>(), jn, delta, lb,
                      j->enc_base + kEncS + (u64)bi * n + (u64)j0, sct.u(), lb);
      } else {
        const Job::EncBatch& e = j->enc_snps.at(bi);
        for (int jj = 0; jj < jn; ++jj) {
          rows.push_back(e.set->view(e.first + j0 + jj));
          pairs[jj].second = rows.back().get();
        }
      }
      CtSet t = T3->slice((int)(bi - b0), 1, lb);
      if (j0 > 0) t.scale = T3->scale;
      set_tensor_mac(c, pairs, jn, t, j0 > 0);
      T3->scale = t.scale;
    }
    if (host) cp->release(ci & 1);
  }
  CtSetPtr Sp = set_new(c, nbt, 2, lb, lb, 1.0);
  set_relin_rescale(c, *T3, *Sp);  // S' at lb - 1
  return Sp;
}

// factored layout (second form of eq. Sprime) for batches [b0, b1):
//   S_i = Enc(CCP batch i) at kFactLevel limbs
//   U_ic = Dup(X_c) S_i; colSum (Alg. 5) puts (X^T S_i)[c, .] at the block heads
//   R_ic = U_ic masked to the heads, broadcast down the block (right ladder)
//   S'_i = S_i - sum_c Dup((XA)_c) R_ic   (tensor sum, relinearise, rescale)
// count CCP SNP batches from b0 into out ([count][2][lf][N]), encryption id
// of batch b = kEncSccp + b
void encrypt_ccp_batches(Job* j, const SnpSrc& src, long b0, int count, u64* out) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  const double delta = std::ldexp(1.0, c->P.scale_bits);
  Tmp z(c, sizeof(double2) * (size_t)count * lay.M);
  build_snp_ccp(c, src.S, src.ld, src.col0, lay.n, lay.k, b0 * lay.tau, count, lay.tau, lay.nb,
                lay.B, lay.M, z.as<double2>());
  encrypt_slots(c, z.as<double2>(), count, delta, kFactLevel, j->enc_base + kEncSccp + (u64)b0,
                out, kFactLevel);
}

CtSetPtr sprime_factored(Job* j, Eval& ev, const SnpSrc* src, long b0, long b1) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  const int d = lay.d, lf = kFactLevel, lb = kBatchLevel;
  const double delta = std::ldexp(1.0, c->P.scale_bits);
  const int nbt = (int)(b1 - b0);
  CtSetPtr Sset = set_new(c, nbt, 2, lf, lf, delta);
  if (src) {
    encrypt_ccp_batches(j, *src, b0, nbt, Sset->d);
  } else {
    // the batches encrypted ahead of the loop, gathered into one set
    for (int i = 0; i < nbt; ++i) {
      const Job::EncBatch& e = j->enc_snps.at(b0 + i);
      GWHE_CUDA(cudaMemcpyAsync(Sset->item(i), e.set->item(e.first), sizeof(u64) * Sset->stride(),
                                cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  std::vector<CtPtr> sv;
  for (int i = 0; i < nbt; ++i) sv.push_back(Sset->view(i));
  // U = Dup(X_c) S_i for all (i, c), item i d + c
  CtSetPtr U = set_new(c, nbt * d, 2, lf, lf, 1.0);
  {
    std::vector<std::pair<const Ct*, const Ct*>> pr;
    for (int i = 0; i < nbt; ++i)
      for (int cc = 0; cc < d; ++cc) pr.push_back({j->DupX[cc].get(), sv[i].get()});
    set_mult(c, pr, *U);
  }
  set_ladder(c, *U, ev.colsum_steps());
  // keep the block heads, then broadcast them down their blocks
  const int lu = U->l;
  const double ql = (double)c->mod[lu - 1];
  auto heads = ev.slots_zero();
  for (int b = 0; b < lay.B; ++b) heads[b * lay.nb] = make_double2(1, 0);
  const u64* hp = mask_pt(c, kMaskHeads, lay.nb, lu, ql, heads);
  std::vector<MaskItem> mi;
  for (int it = 0; it < nbt * d; ++it) mi.push_back(MaskItem{U->item(it), U->cap, hp});
  CtSetPtr R = set_new(c, nbt * d, 2, lu, lu, 1.0);
  set_mask(c, mi, U->scale, ql, *R, true);
  U.reset();
  set_ladder(c, *R, ev.bcast_steps());
  // S'_i = S_i - sum_c Dup((XA)_c) R_ic
  const int lr = R->l;
  std::vector<CtPtr> bv, rv;
  for (int cc = 0; cc < d; ++cc) bv.push_back(ev.view(*j->DupB[cc], lr));
  std::vector<std::pair<const Ct*, const Ct*>> pairs;
  for (int i = 0; i < nbt; ++i)
    for (int cc = 0; cc < d; ++cc) {
      rv.push_back(R->view(i * d + cc));
      pairs.push_back({bv[cc].get(), rv.back().get()});
    }
  CtSetPtr T3 = set_new(c, nbt, 3, lr, lr, 1.0);
  set_tensor_mac(c, pairs, d, *T3);
  R.reset();
  CtSetPtr P = set_new(c, nbt, 2, lr, lr, 1.0);
  set_relin_rescale(c, *T3, *P);
  T3.reset();
  GWHE_REQUIRE(P->l == lb - 1, ST_ELEVEL, "factored S' must leave at kBatchLevel - 1 limbs");
  CtSetPtr Sp = set_new(c, nbt, 2, lb - 1, lb - 1, 1.0);
  Ct sa = Sset->slice(0, nbt, lb - 1).all(), pa = P->all(), oa = Sp->all();
  op_addsub(c, sa, pa, oa, true);
  Sp->scale = Sset->scale;
  return Sp;
}

// S' of every batch encrypted ahead of the loop, in chunks of at most
// kSnpChunk batches from the first batch of each run of consecutive batches:
// the chunks the SNP loop makes of such a run (it uses a chunk whose bounds
// match and computes any other from the encrypted batches, which it keeps
// until consumed)
void precompute_sprime(Job* j, Eval& ev) {
  auto it = j->enc_snps.begin();
  while (it != j->enc_snps.end()) {
    const long c0 = it->first;
    long c1 = c0;
    while (c1 - c0 < kSnpChunk && j->enc_snps.count(c1)) ++c1;
    CtSetPtr sp = sprime_factored(j, ev, nullptr, c0, c1);
    j->sprime_pre[c0] = std::make_pair(c1, std::move(sp));
    it = j->enc_snps.lower_bound(c1);
  }
}

// Runs fn(src, c0, c1) over [b0, b1) in chunks of kSnpChunk batches with the
// chunk's genotype columns on the device.  Genotypes in host memory (the host
// tier) are never copied whole: each chunk's columns go through one of two
// pinned staging buffers (filled by this thread while the device works on the
// previous chunk) and one of two device buffers (filled by a copy stream that
// overlaps the compute stream).
template <class F>
void for_each_snp_chunk(Job* j, const double* S, long b0, long b1, F&& fn) {
  const Layout& lay = j->lay;
  if (is_device_ptr(S)) {
    for (long c0 = b0; c0 < b1; c0 += kSnpChunk)
      fn(SnpSrc{S, lay.k, 0}, c0, std::min(b1, c0 + kSnpChunk));
    return;
  }
  HostStager st(j->c, lay.n, std::min<long>(lay.k, (long)kSnpChunk * lay.tau));
  for (long c0 = b0, i = 0; c0 < b1; c0 += kSnpChunk, ++i) {
    const long c1 = std::min(b1, c0 + kSnpChunk);
    const long col0 = c0 * lay.tau, w = std::min(lay.k, c1 * lay.tau) - col0;
    const double* dev = st.stage((int)(i & 1), S, lay.k, col0, w);
    fn(SnpSrc{dev, w, col0}, c0, c1);
    st.release((int)(i & 1));
  }
}

}  // namespace

void job_encrypt_snps(Job* j, const double* S, long b0, long b1) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  const int n = lay.n, lb = kBatchLevel, lf = kFactLevel;
  const double delta = std::ldexp(1.0, c->P.scale_bits);
  GWHE_REQUIRE(S, ST_EINVAL, "null genotypes");
  GWHE_REQUIRE(0 <= b0 && b0 <= b1 && b1 <= lay.batches, ST_EINVAL, "bad batch range");
  for_each_snp_chunk(j, S, b0, b1, [&](const SnpSrc& src, long c0, long c1) {
    const int nbt = (int)(c1 - c0);
    if (j->factored) {
      std::shared_ptr<CtSet> set(set_new(c, nbt, 2, lf, lf, delta).release());
      encrypt_ccp_batches(j, src, c0, nbt, set->d);
      for (int i = 0; i < nbt; ++i) j->enc_snps[c0 + i] = Job::EncBatch{set, i};
      return;
    }
    // M-CCP: the n REP rows of every batch (encryption id kEncS + b n + row)
    std::shared_ptr<CtSet> set(set_new(c, nbt * n, 2, lb, lb, delta).release());
    Tmp z(c, sizeof(double2) * (size_t)n * lay.M);
    for (long bi = c0; bi < c1; ++bi) {
      const int first = (int)(bi - c0) * n;
      build_snp_rep(c, src.S, src.ld, src.col0, n, lay.k, bi * lay.tau, lay.nb, lay.B, lay.M,
                    z.as<double2>());
      encrypt_slots(c, z.as<double2>(), n, delta, lb, j->enc_base + kEncS + (u64)bi * n,
                    set->item(first), lb);
      j->enc_snps[bi] = Job::EncBatch{set, first};
    }
  });
}

void job_snp_stats(Job* j, const double* S, long b0, long b1) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  Eval ev{c, lay};
  const int n = lay.n;
  if (j->factored)
    GWHE_REQUIRE((int)j->DupX.size() == lay.d && (int)j->DupB.size() == lay.d && j->DupW &&
                     j->DupWZ,
                 ST_EINVAL, "covariate phase not done (fit first)");
  else
    GWHE_REQUIRE((int)j->DupM.size() == n && j->DupW && j->DupWZ, ST_EINVAL,
                 "covariate phase not done (fit or set the fit state first)");
  GWHE_REQUIRE(0 <= b0 && b0 <= b1 && b1 <= lay.batches, ST_EINVAL, "bad batch range");
  if (b0 == b1) return;
  if ((long)j->out.size() < lay.batches) j->out.resize(lay.batches);
  auto run_chunk = [&](const SnpSrc* src, long c0, long c1) {
    if (j->factored)
      batch_body(j, ev, sprime_factored(j, ev, src, c0, c1), c0);
    else
      batch_body(j, ev, sprime_mccp(j, src, c0, c1), c0);
  };
  if (!S) {
    // the batches' ciphertexts from job_encrypt_snps, freed once consumed;
    // a chunk whose S' the fit computed beside the covariate phase goes
    // straight to the batch core
    for (long bi = b0; bi < b1; ++bi)
      GWHE_REQUIRE(j->enc_snps.count(bi), ST_EINVAL,
                   "batch " + std::to_string(bi) + " was not encrypted (gwhe_encrypt_snps)");
    for (long c0 = b0; c0 < b1; c0 += kSnpChunk) {
      const long c1 = std::min(b1, c0 + kSnpChunk);
      auto pre = j->sprime_pre.find(c0);
      if (j->factored && pre != j->sprime_pre.end() && pre->second.first == c1) {
        CtSetPtr sp = std::move(pre->second.second);
        j->sprime_pre.erase(pre);
        batch_body(j, ev, std::move(sp), c0);
      } else {
        run_chunk(nullptr, c0, c1);
      }
      for (long bi = c0; bi < c1; ++bi) j->enc_snps.erase(bi);
    }
    // precomputed chunks that overlap the range but were not used
    for (auto it = j->sprime_pre.begin(); it != j->sprime_pre.end();)
      it = (it->first < b1 && it->second.first > b0) ? j->sprime_pre.erase(it) : std::next(it);
    return;
  }
  for_each_snp_chunk(j, S, b0, b1,
                     [&](const SnpSrc& src, long c0, long c1) { run_chunk(&src, c0, c1); });
}

void job_decrypt(Job* j, double* num, double* den) {
  Context* c = j->c;
  const Layout& lay = j->lay;
  const int N = c->N, M = lay.M;
  std::vector<long> have;
  for (long bi = 0; bi < (long)j->out.size(); ++bi)
    if (j->out[bi][0]) have.push_back(bi);
  GWHE_REQUIRE(!have.empty(), ST_EINVAL, "no batch results to decrypt");
  const int cnt = (int)have.size() * 3;
  Tmp m(c, sizeof(u64) * (size_t)cnt * N);
  {
    // one decryption of every output's q0 limb, then one inverse transform
    GWHE_REQUIRE(c->d_sk, ST_ENOKEY, "no secret key");
    std::vector<const u64*> ptr(2 * (size_t)cnt);
    for (size_t h = 0; h < have.size(); ++h)
      for (int o = 0; o < 3; ++o) {
        const Ct& v = *j->out[have[h]][o];
        ptr[h * 3 + o] = v.poly(0);
        ptr[cnt + h * 3 + o] = v.poly(1);
      }
    Tmp dp(c, sizeof(u64*) * ptr.size());
    GWHE_CUDA(cudaMemcpyAsync(dp.p, ptr.data(), sizeof(u64*) * ptr.size(), cudaMemcpyHostToDevice,
                              c->stream));
    const u64* const* p0 = (const u64* const*)dp.p;
    decrypt_q0_list(c, p0, p0 + cnt, cnt, m.u());
    ntt_inverse(c, m.u(), rows_q(cnt, 1, 1));
  }
  Tmp z(c, sizeof(double2) * (size_t)cnt * M);
  Tmp work(c, sizeof(double2) * (size_t)cnt * M);
  // scales differ per output: decode with scale 1 and divide on the host
  decode_batch(c, m.u(), cnt, 1.0, z.as<double2>(), work.as<double2>());
  // only slot b * nb of each output holds a result: gather those B slots
  const int B = lay.B;
  gather_slots(c, z.as<double2>(), cnt, M, B, lay.nb, work.as<double2>());
  std::vector<double2> hz((size_t)cnt * B);
  GWHE_CUDA(cudaMemcpyAsync(hz.data(), work.p, sizeof(double2) * hz.size(), cudaMemcpyDeviceToHost,
                            c->stream));
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
  for (size_t h = 0; h < have.size(); ++h) {
    const long bi = have[h];
    const double sn = j->out[bi][0]->scale, se = j->out[bi][1]->scale, so = j->out[bi][2]->scale;
    const double2* zn = hz.data() + (h * 3 + 0) * B;
    const double2* ze = hz.data() + (h * 3 + 1) * B;
    const double2* zo = hz.data() + (h * 3 + 2) * B;
    for (int b = 0; b < B; ++b) {
      const long s0 = bi * lay.tau + 2L * b;
      const int slot = b;
      if (s0 < lay.k) {
        num[s0] = zn[slot].x / sn;
        den[s0] = ze[slot].x / se;
      }
      if (s0 + 1 < lay.k) {
        num[s0 + 1] = zn[slot].y / sn;
        den[s0 + 1] = zo[slot].x / so;
      }
    }
  }
}

}  // namespace gwhe
