// server.cu -- continuous batching of encrypted GWAS jobs on one GPU.
//
// A server owns W worker threads.  Each worker has its own CUDA stream and a
// child context of the caller's context, so all workers share one set of
// device-resident evaluation keys and tables while their kernels run on
// separate streams and overlap on the device.  Requests (one GWAS job each:
// n samples, d covariates, k SNPs, host inputs copied at submission) wait in
// arrival order; a free worker admits the first waiting request whose
// estimated device footprint fits in the HBM budget still unclaimed by the
// running jobs, so small jobs flow past a large one that has to wait for
// memory.  A job runs the covariate phase, then its SNP batches in chunks,
// decrypting each chunk and dropping its ciphertexts before the next, which
// bounds its footprint independently of k.  Results are kept until the caller
// collects them.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "capi_types.cuh"
#include "gwas.cuh"

using namespace gwhe;

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  long id = 0;
  int n = 0, d = 0, layout = 0, kappa = 1;
  long k = 0;
  u32 nonce = 0;
  std::vector<double> X, A, y, S;
  const double* S_borrowed = nullptr;  // the caller's genotypes (not copied)
  size_t footprint = 0;
  int dupm_chunk = 0;  // > 0: Dup(M_j) in the host tier
  std::vector<double> num, den;
  int status = GWHE_OK;
  std::string error;
  double t_submit = 0, t_start = 0, t_done = 0;
  // device timeline of the job (ms after the server's reference event)
  double dev_start = 0, dev_end = 0, dev_snp_start = 0, dev_snp_end = 0;
  bool hi = false;  // its SNP loop ran on the worker's high-priority stream
  bool done = false;
};
typedef std::shared_ptr<Request> ReqPtr;

}  // namespace

struct gwhe_server {
  gwhe_ctx* owner = nullptr;
  size_t budget = 0, in_use = 0, peak = 0;
  int chunk = 64;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ReqPtr> pending;
  std::map<long, ReqPtr> reqs;
  long next_id = 1, admitted = 0, running = 0, host_tier = 0, max_running = 0;
  // workers that set up their stream and child context / that failed to
  int live = 0, failed = 0;
  std::string setup_error;
  std::condition_variable cv_setup;
  // one running job at a time holds the high-priority token: its kernels
  // are scheduled first, the others' fill the SMs it leaves idle
  bool hi_taken = false;
  // GWHE_SERVER_ONE_SNP_LOOP: covariate phases run on low-priority streams
  // and the SNP loops one at a time (the token), on high-priority streams
  bool one_snp = false;
  bool snp_busy = false;
  std::condition_variable cv_snp;
  // reference point of the jobs' device timelines (recorded at creation)
  cudaEvent_t t0 = nullptr;
  bool stop = false;
};

namespace {

// Estimated device bytes of one job beyond the shared keys: the two device
// staging buffers of the genotype columns (S itself stays in host memory),
// the encrypted inputs, the covariate phase's largest temporaries and one
// chunk of SNP batches with its outputs.
// (dupm_chunk > 0: the M-CCP layout's Dup(M_j) lives in the host tier and
// only two prefetch slots of dupm_chunk ciphertexts are on the device.)
// columns per prefetched chunk of Dup(M_j) when the server spills it: a
// quarter of the columns, at most 32 (two slots stay well below n columns)
int serve_dupm_chunk(int n) { return std::max(1, std::min(32, n / 4)); }
size_t footprint(const Context* c, int n, int d, long k, bool factored, int chunk,
                 int dupm_chunk = 0) {
  const Layout lay = make_layout(c->logN, n, d, k);
  const double ct = 2.0 * c->N * 8.0;  // bytes per limb of a ciphertext
  const int L = c->P.L;
  const double inputs = (2.0 * d + 2 + (factored ? 0 : (double)d * lay.H)) * L * ct;
  const double fit = ((double)d * d + 6.0 * d + 16) * L * ct * 2.0;
  const long nb = std::min<long>(chunk, lay.batches);
  const double batch = factored ? nb * ((4.0 * d + 8) * kFactLevel + 6.0) * ct * 2.0
                                : ((double)n * kBatchLevel + nb * 16.0) * ct * 2.0 +
                                      (double)n * kBatchLevel * ct;
  const double dupm = dupm_chunk > 0 ? 2.0 * std::min(n, dupm_chunk) * kBatchLevel * ct
                                     : (double)n * (kBatchLevel + 1) * ct;
  const double state = factored ? 2.0 * d * kFactLevel * ct : dupm;
  const long cols = std::min<long>(k, (long)std::min(chunk, 64) * lay.tau);
  const double staging = 2.0 * n * (double)cols * 8;
  return (size_t)(staging + inputs + fit + batch + state);
}

// Worker-owned streams and events of one request's run.
struct RunRes {
  cudaStream_t hi, lo;
  cudaEvent_t t0;        // the server's reference event
  cudaEvent_t s0, s1;    // start / end of the SNP loop
  cudaEvent_t sw;        // stream switch
};

// Holds the server's SNP-loop token for the scope (one_snp servers).
struct SnpToken {
  gwhe_server* srv = nullptr;
  explicit SnpToken(gwhe_server* s) : srv(s) {
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv_snp.wait(lk, [&] { return !srv->snp_busy; });
    srv->snp_busy = true;
  }
  ~SnpToken() {
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->snp_busy = false;
    }
    srv->cv_snp.notify_all();
  }
};

void run_request(gwhe_server* srv, Context* c, Request& r, const RunRes& rr) {
  const int chunk = srv->chunk;
  std::unique_ptr<Job> j(job_create(c, r.n, r.d, r.k, r.layout));
  job_set_nonce(j.get(), r.nonce);
  job_set_host_state(j.get(), r.dupm_chunk);
  job_encrypt_inputs(j.get(), r.X.data(), r.A.data(), r.y.data());
  job_fit(j.get(), r.kappa);
  r.num.assign(r.k, NAN);
  r.den.assign(r.k, NAN);
  std::unique_ptr<SnpToken> token;
  if (srv->one_snp) {
    // the loop runs alone at high priority, ordered after this job's fit
    token.reset(new SnpToken(srv));
    GWHE_CUDA(cudaEventRecord(rr.sw, c->stream));
    GWHE_CUDA(cudaStreamWaitEvent(rr.hi, rr.sw, 0));
    c->stream = rr.hi;
    r.hi = true;
  }
  GWHE_CUDA(cudaEventRecord(rr.s0, c->stream));
  // the genotypes stay in host memory; each chunk's columns are staged
  std::vector<double> num(r.k), den(r.k);
  for (long b0 = 0; b0 < j->lay.batches; b0 += chunk) {
    const long b1 = std::min<long>(j->lay.batches, b0 + chunk);
    job_snp_stats(j.get(), r.S_borrowed ? r.S_borrowed : r.S.data(), b0, b1);
    job_decrypt(j.get(), num.data(), den.data());
    const long s0 = b0 * j->lay.tau, s1 = std::min<long>(r.k, b1 * j->lay.tau);
    for (long s = s0; s < s1; ++s) {
      r.num[s] = num[s];
      r.den[s] = den[s];
    }
    job_release_results(j.get());
  }
  GWHE_CUDA(cudaEventRecord(rr.s1, c->stream));
  GWHE_CUDA(cudaStreamSynchronize(c->stream));
  float a = 0.f, b = 0.f;
  GWHE_CUDA(cudaEventElapsedTime(&a, rr.t0, rr.s0));
  GWHE_CUDA(cudaEventElapsedTime(&b, rr.t0, rr.s1));
  r.dev_snp_start = a;
  r.dev_snp_end = b;
}

void worker_main(gwhe_server* srv) {
  cudaStream_t st = nullptr, st_lo = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr, es0 = nullptr, es1 = nullptr, esw = nullptr;
  Context* c = nullptr;
  try {
    // a new thread starts on device 0: the streams and the child context
    // belong on the owner's device, with its keys and tables
    GWHE_CUDA(cudaSetDevice(srv->owner->c->device));
    int least = 0, greatest = 0;
    GWHE_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    GWHE_CUDA(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest));
    GWHE_CUDA(cudaStreamCreateWithPriority(&st_lo, cudaStreamNonBlocking, least));
    GWHE_CUDA(cudaEventCreate(&e0));
    GWHE_CUDA(cudaEventCreate(&e1));
    GWHE_CUDA(cudaEventCreate(&es0));
    GWHE_CUDA(cudaEventCreate(&es1));
    GWHE_CUDA(cudaEventCreateWithFlags(&esw, cudaEventDisableTiming));
    c = ctx_child(srv->owner->c, st);
  } catch (const std::exception& e) {
    // without a context this worker takes no work; the others carry on
    if (st) cudaStreamDestroy(st);
    if (st_lo) cudaStreamDestroy(st_lo);
    for (cudaEvent_t e : {e0, e1, es0, es1, esw})
      if (e) cudaEventDestroy(e);
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      ++srv->failed;
      srv->setup_error = e.what();
    }
    srv->cv_setup.notify_all();
    return;
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    ++srv->live;
  }
  srv->cv_setup.notify_all();
  for (;;) {
    ReqPtr r;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv_work.wait(lk, [&] {
        if (srv->stop) return true;
        for (auto& p : srv->pending)
          if (p->footprint <= srv->budget - srv->in_use) return true;
        return false;
      });
      if (srv->stop) break;
      for (auto it = srv->pending.begin(); it != srv->pending.end(); ++it)
        if ((*it)->footprint <= srv->budget - srv->in_use) {
          r = *it;
          srv->pending.erase(it);
          break;
        }
      srv->in_use += r->footprint;
      srv->peak = std::max(srv->peak, srv->in_use);
      ++srv->admitted;
      ++srv->running;
      srv->max_running = std::max(srv->max_running, srv->running);
      if (r->dupm_chunk > 0) ++srv->host_tier;
      // without the SNP-loop token, the first job admitted while no other
      // holds it runs on the high-priority stream
      r->hi = !srv->one_snp && !srv->hi_taken;
      if (r->hi) srv->hi_taken = true;
      r->t_start = now_ms();
    }
    // the previous job on this worker has finished on both streams (its
    // run ended with a synchronisation), so switching needs no ordering
    c->stream = r->hi ? st : st_lo;
    const bool held_hi = r->hi;
    try {
      GWHE_CUDA(cudaEventRecord(e0, c->stream));
      run_request(srv, c, *r, RunRes{st, st_lo, srv->t0, es0, es1, esw});
      GWHE_CUDA(cudaEventRecord(e1, c->stream));
      GWHE_CUDA(cudaEventSynchronize(e1));
      float a = 0.f, b = 0.f;
      GWHE_CUDA(cudaEventElapsedTime(&a, srv->t0, e0));
      GWHE_CUDA(cudaEventElapsedTime(&b, srv->t0, e1));
      r->dev_start = a;
      r->dev_end = b;
    } catch (const Error& e) {
      r->status = e.code;
      r->error = e.what();
      cudaStreamSynchronize(c->stream);
    } catch (const std::exception& e) {
      r->status = GWHE_EINVAL;
      r->error = e.what();
      cudaStreamSynchronize(c->stream);
    }
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      if (held_hi) srv->hi_taken = false;
      srv->in_use -= r->footprint;
      --srv->running;
      r->t_done = now_ms();
      r->done = true;
      r->X.clear();
      r->A.clear();
      r->y.clear();
      r->S.clear();
      r->X.shrink_to_fit();
      r->S.shrink_to_fit();
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
  c->stream = st;
  ctx_destroy(c);
  cudaStreamDestroy(st);
  cudaStreamDestroy(st_lo);
  for (cudaEvent_t e : {e0, e1, es0, es1, esw}) cudaEventDestroy(e);
}

}  // namespace

extern "C" {

int gwhe_server_create(gwhe_ctx* ctx, int workers, uint64_t hbm_budget, int chunk_batches,
                       gwhe_server** out) {
  return gwhe_server_create_ex(ctx, workers, hbm_budget, chunk_batches, 0, out);
}

int gwhe_server_create_ex(gwhe_ctx* ctx, int workers, uint64_t hbm_budget, int chunk_batches,
                          int flags, gwhe_server** out) {
  if (!ctx || !ctx->c || !out || workers < 1 || workers > 64 || chunk_batches < 1 ||
      (flags & ~GWHE_SERVER_ONE_SNP_LOOP))
    return GWHE_EINVAL;
  *out = nullptr;
  Context* c = ctx->c;
  if (device_check(c->device, [] {
        int d = -1;
        return cudaGetDevice(&d) == cudaSuccess ? d : -1;
      }()) != ST_OK) {
    c->last_error = "server: the current CUDA device is not the context's device";
    return GWHE_EINVAL;
  }
  if (!c->have_keys) {
    c->last_error = "server: generate the keys first";
    return GWHE_ENOKEY;
  }
  std::unique_ptr<gwhe_server> s(new gwhe_server());
  s->owner = ctx;
  s->chunk = chunk_batches;
  s->one_snp = (flags & GWHE_SERVER_ONE_SNP_LOOP) != 0;
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return GWHE_ECUDA;
    hbm_budget = (uint64_t)(0.6 * (double)fr);
  }
  s->budget = hbm_budget;
  if (cudaEventCreate(&s->t0) != cudaSuccess || cudaEventRecord(s->t0, c->stream) != cudaSuccess ||
      cudaEventSynchronize(s->t0) != cudaSuccess) {
    if (s->t0) cudaEventDestroy(s->t0);
    c->last_error = "server: reference event failed";
    return GWHE_ECUDA;
  }
  for (int w = 0; w < workers; ++w) s->workers.emplace_back(worker_main, s.get());
  {
    // every worker has set up or failed; with none alive, no job could ever
    // run (a submitted job would wait forever), so creation fails
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_setup.wait(lk, [&] { return s->live + s->failed == workers; });
    if (s->live == 0) {
      c->last_error = "server: no worker could set up its stream and context: " + s->setup_error;
      s->stop = true;
      lk.unlock();
      for (auto& t : s->workers) t.join();
      cudaEventDestroy(s->t0);
      return GWHE_ECUDA;
    }
  }
  *out = s.release();
  return GWHE_OK;
}

static int server_submit(gwhe_server* s, int n, int d, long k, int layout, int kappa,
                         uint32_t nonce, const double* X, const double* XtX_inv, const double* y,
                         const double* S, bool borrow, long* id) {
  if (!s || !X || !XtX_inv || !y || !S || !id || n < 1 || d < 1 || k < 1 || kappa < 1)
    return GWHE_EINVAL;
  Context* c = s->owner->c;
  try {
    const Layout lay = make_layout(c->logN, n, d, k);  // rejects shapes that do not fit
    (void)lay;
    if (nonce > kMaxNonce) throw Error(ST_EINVAL, "job nonce out of range");
    if (layout != kLayoutAuto && layout != kLayoutMccp && layout != kLayoutFactored)
      throw Error(ST_EINVAL, "bad layout mode");
  } catch (const Error& e) {
    c->last_error = e.what();
    return e.code;
  }
  auto r = std::make_shared<Request>();
  r->n = n;
  r->d = d;
  r->k = k;
  r->layout = layout;
  r->kappa = kappa;
  r->nonce = nonce;
  r->X.assign(X, X + (size_t)n * d);
  r->A.assign(XtX_inv, XtX_inv + (size_t)d * d);
  r->y.assign(y, y + n);
  if (borrow)
    r->S_borrowed = S;
  else
    r->S.assign(S, S + (size_t)n * k);
  const bool factored =
      layout == kLayoutFactored || (layout == kLayoutAuto && c->P.L > kMLevel);
  r->footprint = footprint(c, n, d, k, factored, s->chunk);
  if (r->footprint > s->budget && !factored) {
    // over the budget with Dup(M_j) on the device: try the host tier
    const size_t fh = footprint(c, n, d, k, false, s->chunk, serve_dupm_chunk(n));
    if (fh <= s->budget) {
      r->footprint = fh;
      r->dupm_chunk = serve_dupm_chunk(n);
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->footprint > s->budget) {
      c->last_error = "server: the job's footprint exceeds the HBM budget";
      return GWHE_ENOMEM;
    }
    r->id = s->next_id++;
    r->t_submit = now_ms();
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    *id = r->id;
  }
  s->cv_work.notify_all();
  return GWHE_OK;
}

int gwhe_server_submit(gwhe_server* s, int n, int d, long k, int layout, int kappa, uint32_t nonce,
                       const double* X, const double* XtX_inv, const double* y, const double* S,
                       long* id) {
  return server_submit(s, n, d, k, layout, kappa, nonce, X, XtX_inv, y, S, false, id);
}

int gwhe_server_submit_borrowed(gwhe_server* s, int n, int d, long k, int layout, int kappa,
                                uint32_t nonce, const double* X, const double* XtX_inv,
                                const double* y, const double* S, long* id) {
  return server_submit(s, n, d, k, layout, kappa, nonce, X, XtX_inv, y, S, true, id);
}

int gwhe_server_wait(gwhe_server* s, long id, double* num, double* den, double* times_ms) {
  if (!s || !num || !den) return GWHE_EINVAL;
  ReqPtr r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return GWHE_EINVAL;
    r = it->second;
    s->cv_done.wait(lk, [&] { return r->done; });
    s->reqs.erase(it);
  }
  if (times_ms) {
    times_ms[0] = r->t_start - r->t_submit;  // waiting for admission
    times_ms[1] = r->t_done - r->t_start;    // on a worker
    times_ms[2] = r->t_done - r->t_submit;   // total latency
    times_ms[3] = r->dev_start;              // device timeline
    times_ms[4] = r->dev_end;
    times_ms[5] = r->hi ? 1.0 : 0.0;
    times_ms[6] = r->dev_snp_start;
    times_ms[7] = r->dev_snp_end;
  }
  if (r->status != GWHE_OK) {
    s->owner->c->last_error = "server job " + std::to_string(id) + ": " + r->error;
    return r->status;
  }
  std::copy(r->num.begin(), r->num.end(), num);
  std::copy(r->den.begin(), r->den.end(), den);
  return GWHE_OK;
}

int gwhe_server_stats(gwhe_server* s, long out[9]) {
  if (!s || !out) return GWHE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out[7] = s->max_running;
  out[8] = s->live;
  out[0] = s->admitted;
  out[1] = s->running;
  out[2] = (long)s->pending.size();
  out[3] = (long)s->in_use;
  out[4] = (long)s->peak;
  out[5] = (long)s->budget;
  out[6] = s->host_tier;
  return GWHE_OK;
}

int gwhe_server_destroy(gwhe_server* s) {
  if (!s) return GWHE_EINVAL;
  {
    // running jobs finish; waiting ones end with an error
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& r : s->pending) {
      r->status = GWHE_EINVAL;
      r->error = "server stopped before the job was admitted";
      r->done = true;
    }
    s->pending.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto& t : s->workers) t.join();
  if (s->t0) cudaEventDestroy(s->t0);
  delete s;
  return GWHE_OK;
}

long gwhe_job_footprint(const gwhe_ctx* ctx, int n, int d, long k, int layout, int chunk_batches) {
  if (!ctx || !ctx->c || n < 1 || d < 1 || k < 1 || chunk_batches < 1) return -1;
  const Context* c = ctx->c;
  try {
    const bool factored =
        layout == kLayoutFactored || (layout == kLayoutAuto && c->P.L > kMLevel);
    return (long)footprint(c, n, d, k, factored, chunk_batches);
  } catch (...) {
    return -1;
  }
}

}  // extern "C"
