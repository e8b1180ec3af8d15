// gwas.cuh -- the encrypted semi-parallel GWAS job (Algorithms 1-11 of the
// paper) on the gwhe evaluator.
#pragma once

#include <array>
#include <map>

#include "ckks.cuh"

namespace gwhe {

// Slot geometry (section "Batching SNPs"): nb = next power of two >= n,
// B = M / nb blocks (complex SNP columns per ciphertext), tau = 2B SNPs per
// batch (eq. numSNPinBatch read as N / nb), H = ceil(n / B) ciphertexts for the
// n x n CCP matrix M.
struct Layout {
  int logN = 0, n = 0, d = 0;
  long k = 0;
  int M = 0, nb = 0, B = 0, tau = 0, H = 0;
  long batches = 0;
};
Layout make_layout(int logN, int n, int d, long k);

constexpr int kBatchLevel = 4;  // limbs with which a SNP batch enters the loop
// M = I - X A X^T is needed only at kBatchLevel + 1 limbs (the Dup(M_j) source):
// it is computed from X and A dropped to this level
constexpr int kMLevel = kBatchLevel + 4;
// factored layout: a CCP SNP batch enters with this many limbs; S' = S - (XA)(X^T S)
// (product, mask, product) leaves at kBatchLevel - 1 like the M-CCP layout's S'
constexpr int kFactLevel = kBatchLevel + 2;

// SNP-phase layouts (both from eq. Sprime): M-CCP = S' = M S with M held as a
// CCP matrix and S as n REP rows per batch; factored = S' = S - (XA)(X^T S)
// with one CCP ciphertext per batch and no n x n matrix.  Auto picks the
// factored layout on rings deep enough for the fit (more than kMLevel limbs)
// and M-CCP otherwise (split mode).
enum LayoutMode { kLayoutAuto = 0, kLayoutMccp = 1, kLayoutFactored = 2 };

struct Job {
  Context* c = nullptr;
  Layout lay;
  std::vector<CtPtr> X, A;
  std::vector<std::vector<CtPtr>> XtREP;  // [d][H]
  CtPtr y, beta0, beta, z, zp, w_m, wzp;
  std::vector<CtPtr> Mct;                 // [H]
  std::vector<CtPtr> DupM;                // [n]      (M-CCP)
  std::vector<CtPtr> DupX, DupB;          // [d] Dup(X_c), Dup((XA)_c) (factored)
  CtPtr DupW, DupWZ;
  bool factored = false;
  u64 enc_base = 0;  // job nonce << 36, added to every encryption id
  std::vector<std::array<CtPtr, 3>> out;  // per batch: num, denEven, denOdd (views)
  std::vector<CtSetPtr> sets;             // storage behind the views above
  // host tier: Dup(M_j) held in pinned host memory (columns per prefetched
  // chunk when dupm_chunk > 0; 0 keeps it on the device)
  int dupm_chunk = 0;
  u64* DupM_host = nullptr;
  bool DupM_host_lent = false;  // DupM_host is the context's pinned block
  // SNP batches encrypted ahead of the loop (job_encrypt_snps): batch b ->
  // items [first, first + per batch) of a shared set (factored: one CCP
  // ciphertext at kFactLevel; M-CCP: the n REP rows at kBatchLevel); a set
  // is freed once the loop has consumed all of its batches
  struct EncBatch {
    std::shared_ptr<CtSet> set;
    int first = 0;
  };
  std::map<long, EncBatch> enc_snps;
  // factored layout: S' of chunks of encrypted batches, computed by the fit
  // beside the covariate phase (S' needs only X, A and S): chunk start ->
  // (chunk end, S' at kBatchLevel - 1 limbs); consumed by the SNP loop
  std::map<long, std::pair<long, CtSetPtr>> sprime_pre;
  ~Job();
};

Job* job_create(Context* c, int n, int d, long k, int mode = kLayoutAuto);
// distinct nonces keep the encryption randomness of jobs under one key apart
constexpr int kNonceShift = 36;
constexpr u32 kMaxNonce = (1u << 12) - 1;
void job_set_nonce(Job* j, u32 nonce);
// drop the kept batch outputs (after they were decrypted)
void job_release_results(Job* j);
// rotation steps whose keys the job needs
std::vector<int> job_rotation_steps(const Job* j);
void job_encrypt_inputs(Job* j, const double* X, const double* A, const double* y);
// the same ciphertexts in two calls: X as CP, (X^T X)^-1 as CP, X^T as REP;
// then y and beta0 = Enc(0)
void job_encrypt_covariates(Job* j, const double* X, const double* A);
void job_encrypt_phenotype(Job* j, const double* y);
// encrypt SNP batches [b0, b1) of S (host or device, n x k row-major) ahead
// of the loop, with the encryption ids the fused loop uses
void job_encrypt_snps(Job* j, const double* S, long b0, long b1);
void job_fit(Job* j, int kappa);
void job_set_fit_state(Job* j, const double* M, const double* w, const double* wz);
// S == nullptr: the batches' ciphertexts from job_encrypt_snps
void job_snp_stats(Job* j, const double* S, long b0, long b1);
// keep Dup(M_j) (M-CCP layout) in pinned host memory, streamed back to the
// device in chunks of `chunk` columns per set of SNP batches; 0 = device
void job_set_host_state(Job* j, int chunk);
// the SNP loop's batch-invariant state (factored: Dup(X_c), Dup((XA)_c);
// M-CCP: Dup(M_j); both: Dup(w), Dup(w z')) as one flat buffer, host or
// device, so that other processes can run batches without the fit
size_t job_state_words(const Job* j);
void job_export_state(const Job* j, u64* buf, size_t words);
void job_import_state(Job* j, const u64* buf, size_t words);
void job_decrypt(Job* j, double* num, double* den);

}  // namespace gwhe
