/*
 * gwhe.h -- C ABI of the GB300 CKKS-RNS engine for the encrypted semi-parallel
 * GWAS of "Achieving GWAS with Homomorphic Encryption" (arXiv 1902.04303).
 *
 * Every function returns an int status: GWHE_OK (0) or a negative code below.
 * No exception crosses this boundary.  The text of the last failure of a
 * context is returned by gwhe_last_error().  All host arrays are owned by the
 * caller and only read/written during the call.  Device work runs on the CUDA
 * stream given at context creation (NULL = the legacy default stream); calls
 * that return host data synchronise that stream.  Handles own their device
 * memory, drawn from the device's stream-ordered memory pool.
 *
 * Data layout.  N = 2^logN is the ring degree, M = N/2 the number of complex
 * slots.  A polynomial over l RNS limbs is uint64[l][N] (limb-major); a
 * ciphertext is uint64[2][l][N] = (c0, c1); limb i is modulo q_i, special
 * limb k modulo p_k.  Host import/export is in the COEFFICIENT domain with
 * residues in [0, q_i); device-resident ciphertexts are kept in the NTT
 * domain.  Complex slot vectors are interleaved (re, im) doubles [M][2].
 *
 * Conventions that the paper leaves open (and that the CPU oracle follows
 * from the same statement):
 *   primes      q0 = largest prime < 2^q0_bits with q = 1 (mod 2N); scale
 *               primes nearest 2^scale_bits, alternately below and above;
 *               special primes the next largest below 2^sp_bits.
 *   randomness  ChaCha20 block function (RFC 8439), key = (seed lo, seed hi,
 *               0,...), nonce = (object lo, object hi, tag), counter = block.
 *               Secret and encryption ephemeral ternary ((w mod 3) - 1, word
 *               k%16 of block k/16); errors centred binomial with eta = 21
 *               (popcounts of the low 21 bits of words 2(k%8), 2(k%8)+1 of
 *               block k/8); uniform residues = 128-bit word of block k/4 mod q.
 *               Objects: secret 1, pk.a 2 (tag = limb), pk.e 3, switching key
 *               (id, digit j): a = 2^40 | id << 8 | j (tag = limb), e = 2^41 |
 *               id << 8 | j; encryption id e: v = 3<<48 | e, e0 = 4<<48 | e,
 *               e1 = 5<<48 | e.  Key id 0 = relinearisation, else the Galois
 *               element.
 *   rescale     floor((C + floor(q_l/2)) / q_l) of the CRT integer C.
 *   key switch  hybrid: digits of alpha = ceil(L/dnum) consecutive q-limbs,
 *               ModUp by fast base conversion (no overflow correction), key
 *               digit j = (-a s + e + P [limb in digit j] s', a), ModDown
 *               (x - Conv([x]_P)) P^-1.
 *   encoding    m(zeta^(5^j)) = scale z_j (zeta = exp(i pi/N)) computed by a
 *               fixed-point radix-2 procedure in exact integer arithmetic:
 *               e = least e >= 0 with 2^e >= max |Re|, |Im| of z (<= 40), F =
 *               61 - log2 M - e; G[bitrev(u_j)] = rint(z_j 2^F) with u_j =
 *               ((5^j mod 2N) - 1)/4; decimation-in-time stages len = 2..M
 *               with twiddles rint(2^62 exp(-2 pi i t/M)); c_k = G[k]
 *               rint(2^62 exp(-pi i k/N)); each complex product formed on 128
 *               bits and rounded as (v + 2^61) >> 62; coefficients k and k+M =
 *               rint((double)Re, Im of c_k * scale / 2^(log2 M + F)).
 *   scales      product -> product of scales; rescale -> / (double)q_last; sums
 *               keep the first operand's scale (relative mismatch > 2^-10 is
 *               GWHE_ESCALE); a real constant c multiplies as rint(c q_last)
 *               and then rescales; a constant added is rint(c scale).
 *   rotation    Rotate(ct, r) moves slot i + r to slot i (Galois 5^r); r < 0
 *               rotates the other way.
 */
#ifndef GWHE_H
#define GWHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GWHE_OK 0
#define GWHE_EINVAL (-1)   /* bad argument, shape or parameter set            */
#define GWHE_ENOMEM (-2)   /* device allocation failed                        */
#define GWHE_ELEVEL (-3)   /* depth exhausted / operands at different levels  */
#define GWHE_ESCALE (-4)   /* operand scales differ by more than 2^-10        */
#define GWHE_ENOKEY (-5)   /* required key (public, relinearisation, Galois) missing */
#define GWHE_ETIMEOUT (-6) /* a bounded device wait expired                   */
#define GWHE_ECUDA (-7)    /* CUDA runtime error (text in gwhe_last_error)    */

typedef struct gwhe_ctx gwhe_ctx;
typedef struct gwhe_ct gwhe_ct;
typedef struct gwhe_job gwhe_job;

/* CKKS parameter set (paper section "Homomorphic Encryption": N, L, p; here in
 * RNS form).  logN in [4, 16]; L q-limbs (1 base prime of q0_bits, L-1 scale
 * primes near 2^scale_bits); K special primes of sp_bits; dnum key digits
 * (1..4, each of ceil(L/dnum) <= 16 limbs). */
typedef struct {
  int logN, L, q0_bits, scale_bits, K, sp_bits, dnum;
} gwhe_params;

/* ------------------------------------------------------------ host only
 * These need no GPU. */
/* RNS basis of the convention above: q[L], p[K]. */
int gwhe_gen_primes(const gwhe_params* prm, uint64_t* q, uint64_t* p);
/* Encoding twiddles W[M/2][2] and T[M][2] (sign -1: encode, +1: decode). */
int gwhe_fft_twiddles(int logN, int sign, double* W, double* T);
/* Batch layout of the semi-parallel GWAS (section "Batching SNPs", eq.
 * numSNPinBatch read as tau = N / nb): out = {nb, B = M/nb, tau = 2B,
 * batches = ceil(k/tau), H = ceil(n/B)}.  GWHE_EINVAL when nb > M. */
int gwhe_layout(int logN, int n, long k, long out[5]);

/* ------------------------------------------------------------ context */
/* Creates a context: primes, NTT / base-conversion / encoding tables on the
 * current CUDA device, which becomes the context's device.  seed keys all
 * randomness.  stream = cudaStream_t (of that device) or NULL.  Every later
 * call on the context (and on its ciphertexts, jobs and child contexts) must
 * be made with that device current, else it returns GWHE_EINVAL and does
 * nothing; gwhe_ctx_destroy switches to it by itself.  On failure *out is
 * NULL and the status says why. */
int gwhe_ctx_create(const gwhe_params* prm, uint64_t seed, void* stream, gwhe_ctx** out);
int gwhe_ctx_destroy(gwhe_ctx* ctx);
/* the context's CUDA device */
int gwhe_ctx_device(const gwhe_ctx* ctx, int* device);
/* The device rule above as a host-only check: GWHE_OK when current_device
 * equals context_device (>= 0), else GWHE_EINVAL.  Needs no GPU. */
int gwhe_device_ok(int context_device, int current_device);
/* Device memory as the library sees it: out = {bytes in use from the
 * device's stream-ordered pool, bytes the pool has reserved, free bytes of
 * the device, total bytes of the device}.  Synchronises nothing. */
int gwhe_mem_info(gwhe_ctx* ctx, uint64_t out[4]);
const char* gwhe_last_error(const gwhe_ctx* ctx);
/* moduli q_0..q_{L-1}, p_0..p_{K-1} (L + K values) */
int gwhe_ctx_moduli(const gwhe_ctx* ctx, uint64_t* out);
int gwhe_sync(gwhe_ctx* ctx);
/* Later calls on ctx (and its jobs and ciphertexts) run on `stream`
 * (cudaStream_t of the context's device, NULL = the legacy default stream).
 * Work already queued on the previous stream stays ordered before them: the
 * new stream waits for it.  Memory the library frees later may have come
 * from the previous stream's pool order; that order is kept by the same
 * wait. */
int gwhe_ctx_set_stream(gwhe_ctx* ctx, void* stream);

/* KeyGen (section "Homomorphic Encryption"): secret, public key, the
 * relinearisation key and one switching key per rotation step in rot_steps
 * and, if conj, for complex conjugation.  Keys stay resident on the device. */
int gwhe_keygen(gwhe_ctx* ctx, const int32_t* rot_steps, size_t nrot, int conj);
/* Key material in the coefficient domain for parity checks: the secret as
 * signed coefficients int64[N]; pk as uint64[2][L][N] (b, a); one family of a
 * switching key (the part used by the switches with k special primes, see
 * gwhe_ks_special) as uint64[dk][2][lmax + k][N], dk = ceil(lmax / alpha),
 * rows q_0..q_{lmax-1} then p_0..p_{k-1}. */
int gwhe_export_secret(gwhe_ctx* ctx, int64_t* s);
int gwhe_export_pk(gwhe_ctx* ctx, uint64_t* pk);
int gwhe_export_ksk(gwhe_ctx* ctx, uint32_t key_id, int k, uint64_t* out);
/* Special primes of a key switch at level l (hybrid key switching is not in
 * the paper; this is the library's reading): *k = the fewest leading special
 * primes p_0..p_{k-1} whose bits (sum of bit lengths minus one) exceed the
 * level's widest digit (sum of its q bit lengths) by 24, or all K when none
 * does; *key_lmax (optional) = the highest level with that count, the levels
 * the key family covers. */
int gwhe_ks_special(const gwhe_ctx* ctx, int l, int* k, int* key_lmax);

/* ------------------------------------------------------------ ciphertexts
 * A handle holds npoly (2, or 3 for a tensor) polynomials with room for cap
 * limbs. */
int gwhe_ct_create(gwhe_ctx* ctx, int npoly, int cap, gwhe_ct** out);
int gwhe_ct_destroy(gwhe_ct* ct);
int gwhe_ct_info(const gwhe_ct* ct, int* npoly, int* l, double* scale);
/* coefficient-domain host array uint64[npoly][l][N] -> handle (l <= cap) */
int gwhe_ct_import(gwhe_ct* ct, const uint64_t* coeffs, int npoly, int l, double scale);
/* handle -> coefficient-domain host array uint64[npoly][l][N] */
int gwhe_ct_export(const gwhe_ct* ct, uint64_t* coeffs);

/* Encode (section "Homomorphic Encryption", phi^-1): z = M complex slots
 * (host, interleaved) -> signed coefficients int64[N] (host). */
int gwhe_encode(gwhe_ctx* ctx, const double* z, double scale, int64_t* coeffs);
/* Encode a batch on the device: z_dev = count x M complex slots (interleaved
 * doubles, device), coeffs_dev = count x N signed coefficients (device). */
int gwhe_encode_batch(gwhe_ctx* ctx, const double* z_dev, int count, double scale,
                      int64_t* coeffs_dev);
/* Encrypt(pk, Encode(z)) at level l with randomness of encryption id enc_id. */
int gwhe_encrypt(gwhe_ctx* ctx, const double* z, double scale, int l, uint64_t enc_id,
                 gwhe_ct* out);
/* Encrypt a given integer plaintext (int64[N] coefficients, host). */
int gwhe_encrypt_coeffs(gwhe_ctx* ctx, const int64_t* m, double scale, int l, uint64_t enc_id,
                        gwhe_ct* out);
/* Decrypt: c0 + c1 s, coefficient domain uint64[l][N] (host). */
int gwhe_decrypt(gwhe_ctx* ctx, const gwhe_ct* ct, uint64_t* m);
/* Decrypt then Decode (the ciphertext is read at its first limb: the value
 * times its scale must stay below q0/2): z = M complex slots (host). */
int gwhe_decrypt_decode(gwhe_ctx* ctx, const gwhe_ct* ct, double* z);

/* ------------------------------------------------------------ arithmetic
 * Section "Homomorphic Encryption" (Add, Mult, Rescale, Rotate) in RNS form.
 * out may alias an input unless stated. */
int gwhe_add(gwhe_ctx* ctx, const gwhe_ct* a, const gwhe_ct* b, gwhe_ct* out);
int gwhe_sub(gwhe_ctx* ctx, const gwhe_ct* a, const gwhe_ct* b, gwhe_ct* out);
int gwhe_negate(gwhe_ctx* ctx, const gwhe_ct* a, gwhe_ct* out);
int gwhe_add_const(gwhe_ctx* ctx, gwhe_ct* ct, double c);
int gwhe_mul_int(gwhe_ctx* ctx, gwhe_ct* ct, int64_t k);
int gwhe_mul_const(gwhe_ctx* ctx, gwhe_ct* ct, double c);           /* consumes a level */
/* slot-wise product with the public vector z (M complex, host) encoded at
 * scale q_last, then rescale (consumes a level) */
int gwhe_mul_mask(gwhe_ctx* ctx, const gwhe_ct* a, const double* z, gwhe_ct* out);
/* tensor (d0, d1, d2) of two ciphertexts; out must have npoly = 3 */
int gwhe_tensor(gwhe_ctx* ctx, const gwhe_ct* a, const gwhe_ct* b, gwhe_ct* out);
/* sum_j tensor(a[j], b[j]) into out (npoly 3): the CP-REP inner loop (Alg. 8) */
int gwhe_tensor_sum(gwhe_ctx* ctx, const gwhe_ct* const* a, const gwhe_ct* const* b, size_t n,
                    gwhe_ct* out);
int gwhe_relin(gwhe_ctx* ctx, const gwhe_ct* t3, gwhe_ct* out);
int gwhe_rescale(gwhe_ctx* ctx, gwhe_ct* ct);                         /* drops q_{l-1} */
int gwhe_mult(gwhe_ctx* ctx, const gwhe_ct* a, const gwhe_ct* b, gwhe_ct* out);
int gwhe_rotate(gwhe_ctx* ctx, const gwhe_ct* a, int steps, gwhe_ct* out); /* out != a */
int gwhe_conjugate(gwhe_ctx* ctx, const gwhe_ct* a, gwhe_ct* out);         /* out != a */
/* out = a + sum_i Rotate(a, steps[i]) for 1 <= nsteps <= 15, the rotations'
 * key switches hoisted: one ModUp of c1, each rotation's automorphism applied
 * to the ModUp digits, the inner products with the rotations' keys summed in
 * the extended basis, one ModDown.  m steps r, 2r, ... of a doubling
 * rotate-and-add ladder (Alg. 1, 4, 5, 7) are the sum over {r, 2r, ...,
 * (2^m - 1) r}; the library's ladders run this way, three steps per sum.
 * More than seven rotations run their inner products in chunks of seven that
 * accumulate before the one ModDown.  out != a; needs the rotations' keys. */
int gwhe_rotate_sum(gwhe_ctx* ctx, const gwhe_ct* a, const int32_t* steps, int nsteps,
                    gwhe_ct* out);
/* gwhe_rotate_sum for count ciphertexts of one level and scale at once (the
 * batched form the library's ladders use): out[i] = a[i] + sum_r Rotate(a[i], r),
 * nsteps <= 15; out[i] != a[j]. */
int gwhe_rotate_sum_batch(gwhe_ctx* ctx, const gwhe_ct* const* a, int count,
                          const int32_t* steps, int nsteps, gwhe_ct* const* out);
/* out[i] = Rotate(a[i], step) for count ciphertexts of one level and scale,
 * as one set (every launch covers all of them), then with rescale != 0 the
 * rescale of each; out[i] != a[j]. */
int gwhe_rotate_batch(gwhe_ctx* ctx, const gwhe_ct* const* a, int count, int32_t step,
                      int rescale, gwhe_ct* const* out);
int gwhe_drop(gwhe_ct* ct, int l);                                          /* keep l limbs */
/* Hybrid key switch of one coefficient-domain polynomial x (uint64[l][N],
 * host) with key key_id: out = uint64[2][l][N] coefficient domain (host). */
int gwhe_keyswitch(gwhe_ctx* ctx, const uint64_t* x, int l, uint32_t key_id, uint64_t* out);
/* Batched forward (inverse = 0) or inverse NTT, in place, over device rows
 * dev[npoly][nlimbs][N]; limb i of every poly is modulo q_i. */
int gwhe_ntt_batch(gwhe_ctx* ctx, uint64_t* dev, int npoly, int nlimbs, int inverse);

/* Key switch without any device allocation, for callers that cannot let the
 * library allocate: a serving process whose device memory is already
 * reserved by its own pool, or a request path where an allocator call could
 * block or synchronise the device.  The paper has no counterpart; this is a
 * deployment variant of gwhe_keyswitch.  x_ntt: device uint64[l][N], NTT
 * domain; out_ntt: device uint64[2][l][N], NTT domain (same arithmetic,
 * bit for bit, as gwhe_keyswitch).  Temporaries live in one static 32 MiB
 * device array (2^22 words) that every GPU loading the library holds until
 * exit; a switch at level l needs (3 l + (ceil(l/alpha) + 2)(l + K)) N words,
 * larger requests return GWHE_EINVAL with the sizes in gwhe_last_error.  The
 * array's address on a device is looked up, its module loaded and its memory
 * committed by gwhe_ctx_create on that device, so the calls themselves
 * reserve nothing; a call with another device current than the context's
 * returns GWHE_EINVAL.  Every call shares the one array, so calls that
 * overlap on the GPU (other streams, other contexts on the same device) race
 * and must be serialised by the caller.  The array keeps the previous call's
 * contents; nothing in it needs to start at zero.  Allocates nothing while
 * the kernel timers (gwhe_prof_enable) are off. */
int gwhe_keyswitch_noalloc(gwhe_ctx* ctx, const uint64_t* x_ntt, int l, uint32_t key_id,
                           uint64_t* out_ntt);

/* ------------------------------------------------------------ GWAS job
 * The paper's problem statement (Alg. 11 inputs / outputs): n samples, d
 * covariates (column 0 = intercept), k SNPs.  Input arrays may be host or
 * device pointers (detected per call). */
int gwhe_job_create(gwhe_ctx* ctx, int n, int d, long k, gwhe_job** out);
/* SNP-phase layout, both from eq. Sprime (section "Semi-Parallel GWAS with
 * Homomorphic Encryption"):
 *   GWHE_LAYOUT_MCCP      S' = M S, M = I - X (X^T X)^-1 X^T held as a CCP
 *                         matrix (ceil(n / B) ciphertexts), S as n REP rows
 *                         per batch at 4 limbs (Alg. 8, Alg. 11)
 *   GWHE_LAYOUT_FACTORED  S' = S - (X (X^T X)^-1)(X^T S), the equation's second
 *                         form: S as ONE CCP ciphertext per batch at 6 limbs,
 *                         no n x n matrix; needs the right-rotation keys
 *                         -2^i for 2^i < nb (see gwhe_job_rotation_steps)
 *   GWHE_LAYOUT_AUTO      factored on rings with more than 8 limbs (deep
 *                         enough for the fit), M-CCP below (split mode);
 *                         M-CCP is bounded by the paper's 256-subject limit
 *                         in spirit (section "Discussion"): its CCP matrix
 *                         and n REP rows per batch grow with n^2
 * Both layouts give the same tau = 2 M / nb SNPs per batch and the same
 * outputs; the factored one needs the fit (no split mode). */
#define GWHE_LAYOUT_AUTO 0
#define GWHE_LAYOUT_MCCP 1
#define GWHE_LAYOUT_FACTORED 2
int gwhe_job_create_ex(gwhe_ctx* ctx, int n, int d, long k, int layout, gwhe_job** out);
int gwhe_job_destroy(gwhe_job* job);
/* out[8] = {M slots, nb, B blocks, tau SNPs per batch, H (CCP ciphertexts of
 * M, 0 when factored), batches, layout (GWHE_LAYOUT_MCCP or _FACTORED), limbs
 * with which a SNP batch is encrypted}. */
int gwhe_job_info(const gwhe_job* job, long out[8]);
/* The rotation steps whose Galois keys the job needs (pass them to
 * gwhe_keygen, with conj = 1): 2^i for i < log2(M), plus -2^i for 2^i < nb in
 * the factored layout.  *count = number of steps; steps may be NULL to query
 * the count, else it must hold cap >= *count entries. */
int gwhe_job_rotation_steps(const gwhe_job* job, int32_t* steps, int cap, int* count);
/* X (n x d, row-major) as CP, (X^T X)^-1 (d x d, row-major; client
 * pre-processing, section "Hessian Matrix Approximation") as CP, X^T as REP,
 * y (n) and beta0 = Enc(0), all at the top level (Alg. 9 / Alg. 11 inputs). */
int gwhe_encrypt_inputs(gwhe_job* job, const double* X, const double* XtX_inv, const double* y);
/* The same ciphertexts as gwhe_encrypt_inputs (same encryption ids, bit for
 * bit) in the two calls of the paper's problem statement (section
 * "Semi-Parallel GWAS with Homomorphic Encryption", the server's inputs):
 * the covariates X (CP), (X^T X)^-1 (CP) and X^T (REP, M-CCP layout only),
 * then the phenotype y with beta0 = Enc(0).  gwhe_encrypt_inputs does both
 * in one batched encoding and encryption. */
int gwhe_encrypt_covariates(gwhe_job* job, const double* X, const double* XtX_inv);
int gwhe_encrypt_phenotype(gwhe_job* job, const double* y);
/* Encrypt SNP batches [b0, b1) of S (n x k row-major genotypes, host or
 * device; streamable: call it for consecutive ranges) ahead of the Alg. 11
 * loop: factored layout one CCP ciphertext per batch at 6 limbs, M-CCP the n
 * REP rows of each batch at 4 limbs, with the encryption ids the fused loop
 * uses, so gwhe_snp_stats(job, NULL, ...) then gives the same ciphertexts bit
 * for bit.  They stay on the device until the loop consumes them: 96 N bytes
 * per batch (factored) or 64 n N bytes per batch (M-CCP).  The fused route
 * (gwhe_snp_stats with S) encrypts each set of 64 batches right before its
 * tensor sums and never holds more than one set.  In the factored layout,
 * batches encrypted before gwhe_fit_covariates get their S' (eq. Sprime,
 * second form, which needs only X, (X^T X)^-1 and S) during the fit, on a
 * second stream beside the covariate phase: 64 N more bytes per batch until
 * the loop consumes it, and the same ciphertexts. */
int gwhe_encrypt_snps(gwhe_job* job, const double* S, long b0, long b1);
/* Alg. 9 (kappa iterations), Alg. 10, eqs. z / M / zprime, then Dup(M_j),
 * Dup(w), Dup(w z') for the batches (Alg. 7, Alg. 8).  Factored layout with
 * batches already encrypted (gwhe_encrypt_snps): also the S' of those
 * batches, in sets of at most 64 consecutive batches from the first of each
 * run; the fit's own chain runs on a stream of the next higher priority so
 * that S' fills the device beside it.  gwhe_snp_stats(job, NULL, b0, b1)
 * uses a set whose bounds match a set of its loop and computes the others
 * from the encrypted batches. */
int gwhe_fit_covariates(gwhe_job* job, int kappa);
/* Split mode for rings without the fit's depth: the client supplies M (n x n,
 * row-major), w and w*z' (n) in plaintext; they are duplicated and encrypted. */
int gwhe_set_fit_state(gwhe_job* job, const double* M, const double* w, const double* wz);
/* Alg. 11 loop for batches [b0, b1): S is n x k row-major genotypes (host or
 * device; the caller keeps ownership), or NULL to take the batches encrypted
 * by gwhe_encrypt_snps (GWHE_EINVAL if one of them was not; each is freed once
 * used).  Batches run in sets of 64.  A host S
 * is never copied whole to the device (the host tier, the counterpart of the
 * paper's cache module, section "Smart Cache Module"): each set's columns are
 * gathered into one of two pinned staging buffers by the calling thread and
 * copied on a second stream while the previous set computes; device memory
 * used for S is 2 n min(k, 64 tau) doubles.  The results do not depend on
 * where S lives.  keep != 0 keeps each batch's output ciphertexts for export. */
int gwhe_snp_stats(gwhe_job* job, const double* S, long b0, long b1, int keep);
/* Decrypt + decode the kept batch outputs: num[k], den[k] (host); b' = num/den,
 * err' = 1/den (eqs. estSNPeffect, estSNPerror). */
int gwhe_decrypt_results(gwhe_job* job, double* num, double* den);
/* Job ciphertexts for parity checks: which = 0 num, 1 denEven, 2 denOdd (index
 * = batch); 3 Dup(M_j) (index j); 4 Dup(w); 5 Dup(w z'); 6 z'; 7 beta; 8 the
 * CCP matrix M (index = ciphertext h); 9 z; 10 the masked weights w;
 * factored layout: 11 Dup(X_c), 12 Dup((X (X^T X)^-1)_c) (index c).  *view
 * is a new handle that does not own the device memory: destroy it with
 * gwhe_ct_destroy, and do not use it after the job is destroyed. */
int gwhe_job_ct(gwhe_job* job, int which, long index, gwhe_ct** view);
/* number of key switches issued on the job's context so far */
long gwhe_job_keyswitches(const gwhe_job* job);

/* Stop sharing randomness between jobs under one key: every encryption id of
 * the job is offset by nonce << 36 (0 <= nonce < 4096).  Call before
 * gwhe_encrypt_inputs; jobs that may both be live under one key need
 * different nonces. */
int gwhe_job_set_nonce(gwhe_job* job, uint32_t nonce);
/* Host tier for the M-CCP layout's n Dup(M_j) ciphertexts (the matrix the
 * paper's cache module keeps on disk, section "Smart Cache Module"): with
 * chunk > 0 they are moved to pinned host memory once computed (call before
 * gwhe_fit_covariates / gwhe_set_fit_state), and every set of 64 SNP batches
 * prefetches them back chunk columns at a time into two device slots on a
 * copy stream, each chunk serving all batches of the set.  Device memory for
 * Dup(M_j) drops from n to 2 chunk ciphertexts; results are unchanged (the
 * tensor sums are exact).  chunk = 0 keeps them on the device (default).
 * GWHE_EINVAL for chunk < 0, or to turn the tier off once it holds them. */
int gwhe_job_set_host_state(gwhe_job* job, int chunk);
/* The SNP loop's batch-invariant state, computed by the covariate phase
 * (factored layout: Dup(X_c) and Dup((X (X^T X)^-1)_c) for c < d; M-CCP:
 * Dup(M_j) for j < n; both: Dup(w), Dup(w z'), the inputs of the Alg. 11 loop),
 * as one flat buffer of *words uint64 (host or device memory, caller-owned):
 * a 7-word header (magic, version, N, layout, n, d, count), each
 * ciphertext's level and scale, then its NTT-domain residues [2][l][N].
 * A process holding the same context (parameters, seed, keys) imports it
 * into a job of the same shape and layout and runs SNP batches with no fit
 * of its own: the batches' ciphertexts are bit for bit those of the
 * exporting job.  This is the one broadcast that shards a job's batches over
 * GPUs (section "Batching SNPs": the batches are independent once the state
 * exists).  export: GWHE_EINVAL before the fit or into too small a buffer;
 * import: GWHE_EINVAL if the header does not match the job. */
int gwhe_job_state_size(const gwhe_job* job, size_t* words);
int gwhe_job_export_state(const gwhe_job* job, uint64_t* buf, size_t words);
int gwhe_job_import_state(gwhe_job* job, const uint64_t* buf, size_t words);
/* Drop the kept batch outputs (after gwhe_decrypt_results), so that a long
 * job can evaluate and decrypt its SNP batches chunk by chunk. */
int gwhe_job_release_results(gwhe_job* job);
/* Estimated device bytes of one job beyond the shared keys (the two staging
 * buffers of host genotypes, encrypted inputs, the covariate phase's
 * temporaries, one chunk of chunk_batches SNP batches and its outputs); -1 on
 * bad arguments. */
long gwhe_job_footprint(const gwhe_ctx* ctx, int n, int d, long k, int layout, int chunk_batches);

/* ------------------------------------------------------------ serving
 * Continuous batching of GWAS jobs on one GPU (no counterpart in the paper,
 * which runs one job).  `workers` threads each own two CUDA streams (the
 * device's highest and lowest priority) and a child context sharing ctx's
 * tables and device-resident keys (generated first, with every rotation the
 * jobs need), so jobs overlap on the device.  One running job at a time holds
 * the high-priority stream: its kernels are scheduled first and the other
 * running jobs' kernels fill the SMs it leaves idle.  A free
 * worker admits the first waiting job whose estimated footprint
 * (gwhe_job_footprint) fits in hbm_budget bytes minus the running jobs'
 * (hbm_budget 0 = 60% of the free device memory); a job runs the covariate
 * phase, then its SNP batches chunk_batches at a time, decrypting and
 * dropping each chunk.  Do not use ctx for other work while the server runs;
 * destroy the server before ctx.
 *   submit: copies the host inputs (X n x d row-major, (X^T X)^-1 d x d, y n,
 *           S n x k row-major; S stays in host memory and is staged per set
 *           of batches, see gwhe_snp_stats).  An M-CCP job whose footprint
 *           exceeds the budget with Dup(M_j) on the device runs with it in
 *           the host tier (gwhe_job_set_host_state, min(32, n/4) columns per
 *           chunk) if that fits; ENOMEM if neither fits.
 *   wait:   blocks until the job is done; num[k], den[k] as
 *           gwhe_decrypt_results; times_ms (optional, 8 entries) =
 *           {waiting for admission, running, total (host clock, ms), start
 *           and end of the job's work on the device and start and end of
 *           its SNP loop there (ms after the server's creation, device
 *           clock, entries 3, 4, 6, 7), 1 if its SNP loop ran on the
 *           high-priority stream (entry 5)}; the job's status is returned
 *           and the job is forgotten.
 *   stats:  {admitted, running, waiting, bytes claimed, peak bytes claimed,
 *           budget, jobs run with Dup(M_j) in the host tier, most jobs
 *           running at once, workers alive}.
 *   destroy: running jobs finish, waiting ones end with GWHE_EINVAL.
 * Creation waits until every worker has set up its stream and child context
 * (on ctx's device); if none could, it returns GWHE_ECUDA with the reason in
 * gwhe_last_error(ctx) rather than a server that would never run a job. */
typedef struct gwhe_server gwhe_server;
int gwhe_server_create(gwhe_ctx* ctx, int workers, uint64_t hbm_budget, int chunk_batches,
                       gwhe_server** out);
/* flags: GWHE_SERVER_ONE_SNP_LOOP makes the jobs' covariate phases run on
 * the low-priority streams and their SNP loops one at a time (a job waits
 * after its fit until no other loop runs), each loop on its worker's
 * high-priority stream: a loop saturates the GPU by itself, two of them only
 * contend, while the covariate phases' small launches fill the SMs a loop
 * leaves idle.  Without the flag the priority goes as described above. */
#define GWHE_SERVER_ONE_SNP_LOOP 1
int gwhe_server_create_ex(gwhe_ctx* ctx, int workers, uint64_t hbm_budget, int chunk_batches,
                          int flags, gwhe_server** out);
int gwhe_server_submit(gwhe_server* s, int n, int d, long k, int layout, int kappa, uint32_t nonce,
                       const double* X, const double* XtX_inv, const double* y, const double* S,
                       long* id);
/* As gwhe_server_submit, but S (host memory) is not copied: the caller keeps
 * it alive and unchanged until gwhe_server_wait has returned for this job
 * (the genotype matrix of a large job is gigabytes; its copy would run on
 * the submitting thread). */
int gwhe_server_submit_borrowed(gwhe_server* s, int n, int d, long k, int layout, int kappa,
                                uint32_t nonce, const double* X, const double* XtX_inv,
                                const double* y, const double* S, long* id);
int gwhe_server_wait(gwhe_server* s, long id, double* num, double* den, double* times_ms);
int gwhe_server_stats(gwhe_server* s, long out[9]);
int gwhe_server_destroy(gwhe_server* s);

/* Child context on another stream (void* = cudaStream_t) that shares ctx's
 * tables and keys read-only: for callers that drive several jobs from
 * several threads.  Keys must exist; no key generation on the child; destroy
 * it before ctx. */
int gwhe_ctx_create_child(gwhe_ctx* ctx, void* stream, gwhe_ctx** out);

/* ------------------------------------------------------------ autotuning
 * The N = 2^16 transform is compiled in seven shapes: 0-5 in two launches
 * (passes of 8 + 8, 7 + 9 or 9 + 7 stages; 16 residues per thread in 64-,
 * 128- or 256-thread CTAs, or 32 in 128-thread CTAs), 6 in one launch on a
 * cluster of eight 512-thread CTAs whose distributed shared memory carries
 * the residues between the column and the row stages (each limb read from and
 * written to HBM once); every shape computes identical residues.
 * Launches of fewer than 128 rows (a few waves of CTAs or less, as in the
 * covariate phase's single-ciphertext operations) and larger launches each
 * have their own shape.  gwhe_autotune times a forward and an inverse
 * transform of `rows` rows in each shape on the context's stream, keeps the
 * fastest for launches of that size class (rows < 128 or >= 128; for this
 * context and the child contexts made after it) and returns the times (ms[7],
 * may be NULL) and the choice.  Other ring degrees have one shape (ms all 0).
 * gwhe_set_ntt_variant selects a shape directly (0..6) for both classes; a
 * context starts with shape 4 (8 + 8 x 16 in 128-thread CTAs, the fastest
 * measured on GB300). */
int gwhe_autotune(gwhe_ctx* ctx, int rows, double* ms, int* chosen);
int gwhe_set_ntt_variant(gwhe_ctx* ctx, int variant);

/* ------------------------------------------------------------ instrumentation */
/* key switches issued so far per level: out[l] for l < n */
int gwhe_ks_histogram(const gwhe_ctx* ctx, long* out, int n);
/* number of kernels the context has launched so far */
long gwhe_launch_count(const gwhe_ctx* ctx);
/* Kernel-class timers: when on, CUDA events on the context's stream bracket
 * every launch group of a class; enabling (or disabling) discards earlier
 * records.  Classes: 0 NTT/iNTT, 1 key-switch inner product, 2 tensor sum,
 * 3 base conversion, 4 element-wise, 5 encoding FFT, 6 sampling/encryption. */
#define GWHE_PROF_NCAT 7
int gwhe_prof_enable(gwhe_ctx* ctx, int on);
/* per class since the last read: total event time (ms), algorithmic bytes
 * moved (each input and output residue counted once), launch groups.
 * Synchronises the stream. */
int gwhe_prof_read(gwhe_ctx* ctx, double* ms, double* bytes, long* count);

/* Arithmetic ceiling of the NTT butterfly: runs the transform's Cooley-Tukey
 * butterfly (Shoup product + Harvey lazy corrections, section "Homomorphic
 * Encryption" ring arithmetic) on register-resident residues on every SM, no
 * memory traffic, rounds x 32 butterflies per thread.  *per_s = butterflies
 * per second, *ms (optional) = the timed launch.  Measurement only; the
 * paper has no counterpart. */
int gwhe_probe_butterflies(gwhe_ctx* ctx, int rounds, double* per_s, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* GWHE_H */
