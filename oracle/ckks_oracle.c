/*
 * ckks_oracle.c -- O1: a plain, slow, scalar CPU implementation of textbook
 * RNS-CKKS, written from the scheme's definition (paper section
 * "Homomorphic Encryption": KeyGen, Encrypt, Decrypt, Add, Mult, Rescale,
 * Encode/Decode, Rotate) in its residue-number-system form.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant generator with
 * the CUDA library: every constant here is recomputed from its definition.
 *
 * Style: every modular product is ((unsigned __int128)a * b) % m; every
 * polynomial product is a textbook psi-twisted cyclic NTT (itself pinned
 * against schoolbook negacyclic convolution).  Polynomials are held in the
 * COEFFICIENT domain, limb-major: poly[limb][coefficient].
 *
 * Conventions the paper leaves open (each is one reading, stated once here
 * and mirrored, from the same statement, by the CUDA library):
 *   - primes: q0 = largest prime < 2^q0_bits with q = 1 mod 2N; scale primes
 *     closest to 2^scale_bits, alternately just below and just above it;
 *     special primes = next largest primes < 2^sp_bits, skipping used ones.
 *   - randomness: ChaCha20 block function (RFC 8439) keyed by the seed,
 *     nonce = (object id, tag); ternary secret/ephemeral, centred binomial
 *     error (eta = 21), uniform residues from 128-bit words mod q.
 *   - rescale rounds half up: floor((C + floor(q_l/2)) / q_l).
 *   - hybrid key switching: digits of alpha consecutive q-limbs; ModUp by
 *     fast base conversion without overflow correction; ModDown as
 *     (x - Conv([x]_P)) * P^-1.
 *   - encoding: the fixed-point radix-2 FFT procedure documented at or_encode().
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

#define OR_MAXMOD 128

/* Independent limbs, polynomials and coefficients may be computed by several
 * host threads (OpenMP when the compiler has it).  Every output is computed by
 * one thread in the same order as the serial loop, so results do not depend
 * on the thread count. */
#ifdef _OPENMP
#include <omp.h>
#define OR_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#define OR_PARALLEL_FOR_COLLAPSE2 _Pragma("omp parallel for collapse(2) schedule(static)")
#else
#define OR_PARALLEL_FOR
#define OR_PARALLEL_FOR_COLLAPSE2
#endif

/* number of host threads the loops above use (1 without OpenMP) */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* scalar modular arithmetic                                            */
/* ------------------------------------------------------------------ */
static u64 mmul(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
static u64 madd(u64 a, u64 b, u64 m) { return (u64)(((u128)a + b) % m); }
static u64 msub(u64 a, u64 b, u64 m) { return (u64)(((u128)a + m - (b % m)) % m); }
static u64 mpow(u64 a, u64 e, u64 m)
{
    u64 r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mmul(r, a, m);
        a = mmul(a, a, m);
        e >>= 1;
    }
    return r;
}
/* inverse modulo a prime (Fermat) */
static u64 minv(u64 a, u64 m) { return mpow(a % m, m - 2, m); }
/* signed integer -> residue in [0, m) */
static u64 mred_i64(i64 v, u64 m)
{
    if (v >= 0) return (u64)v % m;
    u64 mag = (u64)(-(v + 1)) + 1u; /* |v| without overflow */
    u64 r = mag % m;
    return r ? m - r : 0;
}

/* ------------------------------------------------------------------ */
/* primality and prime generation                                       */
/* ------------------------------------------------------------------ */
/* Deterministic Miller-Rabin for 64-bit integers (the first twelve prime
 * bases suffice for every n < 3.3e24). */
int or_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n % bases[i] == 0) return n == bases[i];
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        u64 x = mpow(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mmul(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

static int used_in(u64 c, const u64 *list, int n)
{
    for (int i = 0; i < n; i++) if (list[i] == c) return 1;
    return 0;
}

/* Generates the RNS basis.  q[0] is the base prime, q[1..L-1] the scale
 * primes (in the order they are dropped last-to-first), p[0..K-1] the
 * special primes.  Returns 0 on success, -1 if a search runs out. */
int or_gen_primes(int logN, int L, int q0_bits, int scale_bits, int K, int sp_bits,
                  u64 *q, u64 *p)
{
    const u64 step = (u64)2 << logN; /* 2N */
    u64 used[OR_MAXMOD];
    int nused = 0;
    if (L < 1 || L + K > OR_MAXMOD) return -1;
    if (q0_bits > 61 || sp_bits > 61 || scale_bits > 61) return -1;
    /* base prime: largest prime below 2^q0_bits, = 1 mod 2N */
    u64 c = ((u64)1 << q0_bits) + 1 - step;
    while (!or_is_prime(c)) { if (c <= step) return -1; c -= step; }
    q[0] = c; used[nused++] = c;
    /* scale primes: alternate the nearest candidates below and above 2^sb */
    u64 below = ((u64)1 << scale_bits) + 1 - step;
    u64 above = ((u64)1 << scale_bits) + 1;
    for (int i = 1; i < L; i++) {
        if (i % 2 == 1) {
            while (!or_is_prime(below) || used_in(below, used, nused)) {
                if (below <= step) return -1;
                below -= step;
            }
            q[i] = below; below -= step;
        } else {
            while (!or_is_prime(above) || used_in(above, used, nused)) above += step;
            q[i] = above; above += step;
        }
        used[nused++] = q[i];
    }
    /* special primes: next largest below 2^sp_bits, skipping used ones */
    u64 s = ((u64)1 << sp_bits) + 1 - step;
    for (int k = 0; k < K; k++) {
        while (!or_is_prime(s) || used_in(s, used, nused)) {
            if (s <= step) return -1;
            s -= step;
        }
        p[k] = s; used[nused++] = s; s -= step;
    }
    return 0;
}

/* smallest-base primitive 2N-th root of unity mod q (psi^N = -1) */
u64 or_primitive_root_2n(u64 q, int logN)
{
    const u64 twoN = (u64)2 << logN;
    const u64 N = (u64)1 << logN;
    for (u64 x = 2; x < q; x++) {
        u64 r = mpow(x, (q - 1) / twoN, q);
        if (mpow(r, N, q) == q - 1) return r;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* textbook negacyclic polynomial product                               */
/* ------------------------------------------------------------------ */
/* cyclic NTT of length n (power of two): A[k] = sum_j a[j] w^(jk), in place */
static void ntt_cyclic(u64 *a, int n, u64 w, u64 q)
{
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        u64 wl = mpow(w, (u64)(n / len), q);
        for (int i = 0; i < n; i += len) {
            u64 wk = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j];
                u64 v = mmul(a[i + j + len / 2], wk, q);
                a[i + j] = madd(u, v, q);
                a[i + j + len / 2] = msub(u, v, q);
                wk = mmul(wk, wl, q);
            }
        }
    }
}

/* out = a * b mod (X^N + 1, q) using psi-twisted cyclic NTT; out may alias */
void or_polymul(const u64 *a, const u64 *b, u64 *out, int logN, u64 q, u64 psi)
{
    const int N = 1 << logN;
    u64 *A = (u64 *)malloc(sizeof(u64) * N);
    u64 *B = (u64 *)malloc(sizeof(u64) * N);
    u64 pk = 1;
    for (int k = 0; k < N; k++) {
        A[k] = mmul(a[k] % q, pk, q);
        B[k] = mmul(b[k] % q, pk, q);
        pk = mmul(pk, psi, q);
    }
    u64 w = mmul(psi, psi, q);
    ntt_cyclic(A, N, w, q);
    ntt_cyclic(B, N, w, q);
    for (int k = 0; k < N; k++) A[k] = mmul(A[k], B[k], q);
    ntt_cyclic(A, N, minv(w, q), q);
    u64 ninv = minv((u64)N, q), psiinv = minv(psi, q), pinv = 1;
    for (int k = 0; k < N; k++) {
        out[k] = mmul(mmul(A[k], pinv, q), ninv, q);
        pinv = mmul(pinv, psiinv, q);
    }
    free(A);
    free(B);
}

/* schoolbook negacyclic convolution (the definition; used to pin polymul) */
void or_polymul_schoolbook(const u64 *a, const u64 *b, u64 *out, int logN, u64 q)
{
    const int N = 1 << logN;
    u64 *acc = (u64 *)calloc(N, sizeof(u64));
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            u64 t = mmul(a[i] % q, b[j] % q, q);
            int k = i + j;
            if (k < N) acc[k] = madd(acc[k], t, q);
            else acc[k - N] = msub(acc[k - N], t, q);
        }
    memcpy(out, acc, sizeof(u64) * N);
    free(acc);
}

/* ------------------------------------------------------------------ */
/* ChaCha20 block function (RFC 8439, section 2.3)                      */
/* ------------------------------------------------------------------ */
static u32 rotl32(u32 x, int n) { return (x << n) | (x >> (32 - n)); }
static void quarter(u32 *s, int a, int b, int c, int d)
{
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 16);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 12);
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 8);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 7);
}
void or_chacha20_block(const u32 key[8], u32 counter, const u32 nonce[3], u32 out[16])
{
    u32 init[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                    key[0], key[1], key[2], key[3], key[4], key[5], key[6], key[7],
                    counter, nonce[0], nonce[1], nonce[2]};
    u32 s[16];
    memcpy(s, init, sizeof s);
    for (int r = 0; r < 10; r++) {
        quarter(s, 0, 4, 8, 12); quarter(s, 1, 5, 9, 13);
        quarter(s, 2, 6, 10, 14); quarter(s, 3, 7, 11, 15);
        quarter(s, 0, 5, 10, 15); quarter(s, 1, 6, 11, 12);
        quarter(s, 2, 7, 8, 13); quarter(s, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) out[i] = s[i] + init[i];
}

/* one block of the stream (seed, object, tag) */
static void stream_block(u64 seed, u64 obj, u32 tag, u32 counter, u32 out[16])
{
    u32 key[8] = {(u32)seed, (u32)(seed >> 32), 0, 0, 0, 0, 0, 0};
    u32 nonce[3] = {(u32)obj, (u32)(obj >> 32), tag};
    or_chacha20_block(key, counter, nonce, out);
}

/* ternary: coefficient k takes word k%16 of block k/16; value (w mod 3) - 1 */
void or_sample_ternary(u64 seed, u64 obj, int logN, i64 *out)
{
    const int N = 1 << logN;
    u32 blk[16];
    for (int k = 0; k < N; k++) {
        if (k % 16 == 0) stream_block(seed, obj, 0, (u32)(k / 16), blk);
        out[k] = (i64)(blk[k % 16] % 3u) - 1;
    }
}

static int popc21(u32 x)
{
    x &= 0x1FFFFFu;
    int c = 0;
    while (x) { c += (int)(x & 1u); x >>= 1; }
    return c;
}

/* centred binomial, eta = 21: coefficient k uses words 2(k%8), 2(k%8)+1 of
 * block k/8; value popcount(low 21 bits of the first) - popcount(... second) */
void or_sample_cbd(u64 seed, u64 obj, int logN, i64 *out)
{
    const int N = 1 << logN;
    u32 blk[16];
    for (int k = 0; k < N; k++) {
        if (k % 8 == 0) stream_block(seed, obj, 0, (u32)(k / 8), blk);
        int r = k % 8;
        out[k] = (i64)popc21(blk[2 * r]) - (i64)popc21(blk[2 * r + 1]);
    }
}

/* uniform residue mod m: coefficient k uses the 128-bit little-endian word
 * made of words 4(k%4)..4(k%4)+3 of block k/4 of stream (obj, tag) */
void or_sample_uniform(u64 seed, u64 obj, u32 tag, u64 m, int logN, u64 *out)
{
    const int N = 1 << logN;
    u32 blk[16];
    for (int k = 0; k < N; k++) {
        if (k % 4 == 0) stream_block(seed, obj, tag, (u32)(k / 4), blk);
        int r = k % 4;
        u128 x = (u128)blk[4 * r] | ((u128)blk[4 * r + 1] << 32) |
                 ((u128)blk[4 * r + 2] << 64) | ((u128)blk[4 * r + 3] << 96);
        out[k] = (u64)(x % m);
    }
}

/* ------------------------------------------------------------------ */
/* context                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    int logN, N, L, K, alpha, dnum;
    u64 seed;
    u64 mod[OR_MAXMOD]; /* mod[0..L) = q_i, mod[L..L+K) = p_k */
    u64 psi[OR_MAXMOD];
    int ks_k[OR_MAXMOD + 1]; /* special primes used by a key switch at level l */
} or_ctx;

static int bitlen(u64 x)
{
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}

/* Special primes of a key switch at level l (hybrid key switching, a reading
 * of the paper's relinearisation/rotation keys): the fewest leading special
 * primes p_0..p_{k-1} whose product P_k has at least OR_KS_MARGIN more bits
 * than the widest digit at that level, or all K when no count reaches the
 * margin.  Bit counts are bounded from below for P_k (sum of bitlen(p) - 1)
 * and from above for the digits (sum of bitlen(q)), so the rule is
 * integer-only. */
#define OR_KS_MARGIN 24
static int ks_special_rule(const or_ctx *c, int l)
{
    int need = 0;
    for (int lo = 0; lo < l; lo += c->alpha) {
        int hi = lo + c->alpha < l ? lo + c->alpha : l, bits = 0;
        for (int i = lo; i < hi; i++) bits += bitlen(c->mod[i]);
        if (bits > need) need = bits;
    }
    need += OR_KS_MARGIN;
    int have = 0;
    for (int k = 1; k <= c->K; k++) {
        have += bitlen(c->mod[c->L + k - 1]) - 1;
        if (have >= need) return k;
    }
    return c->K;
}

void *or_ctx_create(int logN, int L, int q0_bits, int scale_bits, int K, int sp_bits,
                    int dnum, u64 seed)
{
    if (dnum < 1 || dnum > L || K < 1) return NULL;
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->logN = logN; c->N = 1 << logN; c->L = L; c->K = K; c->dnum = dnum;
    c->alpha = (L + dnum - 1) / dnum;
    c->seed = seed;
    if (or_gen_primes(logN, L, q0_bits, scale_bits, K, sp_bits, c->mod, c->mod + L)) {
        free(c);
        return NULL;
    }
    for (int i = 0; i < L + K; i++) c->psi[i] = or_primitive_root_2n(c->mod[i], logN);
    for (int l = 1; l <= L; l++) c->ks_k[l] = ks_special_rule(c, l);
    return c;
}
int or_ks_special(const void *ctx, int l)
{
    const or_ctx *c = (const or_ctx *)ctx;
    return (l >= 1 && l <= c->L) ? c->ks_k[l] : 0;
}
void or_ctx_destroy(void *ctx) { free(ctx); }
int or_ctx_alpha(const void *ctx) { return ((const or_ctx *)ctx)->alpha; }
void or_ctx_moduli(const void *ctx, u64 *out)
{
    const or_ctx *c = (const or_ctx *)ctx;
    memcpy(out, c->mod, sizeof(u64) * (c->L + c->K));
}

/* object ids of the random streams */
#define OBJ_SK 1ull
#define OBJ_PK_A 2ull
#define OBJ_PK_E 3ull
#define OBJ_KSK_A(key, k, j) ((1ull << 40) | ((u64)(k) << 32) | ((u64)(key) << 8) | (u64)(j))
#define OBJ_KSK_E(key, k, j) ((2ull << 40) | ((u64)(k) << 32) | ((u64)(key) << 8) | (u64)(j))
#define OBJ_ENC_V(id) ((3ull << 48) | (u64)(id))
#define OBJ_ENC_E0(id) ((4ull << 48) | (u64)(id))
#define OBJ_ENC_E1(id) ((5ull << 48) | (u64)(id))

/* secret key s as signed integers (ternary) */
void or_keygen_sk(const void *ctx, i64 *s)
{
    const or_ctx *c = (const or_ctx *)ctx;
    or_sample_ternary(c->seed, OBJ_SK, c->logN, s);
}

/* reduce a signed polynomial into residues for moduli mod[0..n) */
static void signed_to_rns(const or_ctx *c, const i64 *v, const u64 *mods, int n, u64 *out)
{
    for (int u = 0; u < n; u++)
        for (int k = 0; k < c->N; k++) out[(size_t)u * c->N + k] = mred_i64(v[k], mods[u]);
}

/* public key: b = -a s + e (mod q_i), a uniform; b, a are [L][N] */
void or_keygen_pk(const void *ctx, u64 *b, u64 *a)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N;
    i64 *s = (i64 *)malloc(sizeof(i64) * N), *e = (i64 *)malloc(sizeof(i64) * N);
    or_keygen_sk(ctx, s);
    or_sample_cbd(c->seed, OBJ_PK_E, c->logN, e);
    OR_PARALLEL_FOR
    for (int i = 0; i < c->L; i++) {
        u64 q = c->mod[i];
        u64 *sr = (u64 *)malloc(sizeof(u64) * N), *t = (u64 *)malloc(sizeof(u64) * N);
        u64 *ai = a + (size_t)i * N, *bi = b + (size_t)i * N;
        or_sample_uniform(c->seed, OBJ_PK_A, (u32)i, q, c->logN, ai);
        for (int k = 0; k < N; k++) sr[k] = mred_i64(s[k], q);
        or_polymul(ai, sr, t, c->logN, q, c->psi[i]);
        for (int k = 0; k < N; k++) bi[k] = madd(msub(0, t[k], q), mred_i64(e[k], q), q);
        free(sr); free(t);
    }
    free(s); free(e);
}

/* Switching key from target t (residues over all L+K moduli, [L+K][N]) to s,
 * for the key switches that use k special primes, up to level lmax.  Its
 * moduli are q_0..q_{lmax-1} then p_0..p_{k-1} (nm = lmax + k rows) and its
 * digits are the alpha-limb groups of [0, lmax):  out is [dk][2][nm][N],
 * dk = ceil(lmax / alpha); digit j holds b_j = -a_j s + e_j + [u in digit j]
 * P_k t and a_j (uniform).  key_id 0 = relinearisation, otherwise the Galois
 * element. */
void or_keygen_ksk(const void *ctx, u32 key_id, int k, int lmax, const u64 *target, u64 *out)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N, nm = lmax + k, dk = (lmax + c->alpha - 1) / c->alpha;
    i64 *s = (i64 *)malloc(sizeof(i64) * N), *e = (i64 *)malloc(sizeof(i64) * N);
    or_keygen_sk(ctx, s);
    for (int j = 0; j < dk; j++) {
        or_sample_cbd(c->seed, OBJ_KSK_E(key_id, k, j), c->logN, e);
        int lo = j * c->alpha, hi = lo + c->alpha < lmax ? lo + c->alpha : lmax;
        OR_PARALLEL_FOR
        for (int u = 0; u < nm; u++) {
            u64 *sr = (u64 *)malloc(sizeof(u64) * N), *t = (u64 *)malloc(sizeof(u64) * N);
            int gm = u < lmax ? u : c->L + (u - lmax); /* index into mod[] */
            u64 m = c->mod[gm];
            u64 *bj = out + (((size_t)j * 2 + 0) * nm + u) * N;
            u64 *aj = out + (((size_t)j * 2 + 1) * nm + u) * N;
            or_sample_uniform(c->seed, OBJ_KSK_A(key_id, k, j), (u32)gm, m, c->logN, aj);
            for (int kk = 0; kk < N; kk++) sr[kk] = mred_i64(s[kk], m);
            or_polymul(aj, sr, t, c->logN, m, c->psi[gm]);
            u64 Pm = 1;
            for (int kk = 0; kk < k; kk++) Pm = mmul(Pm, c->mod[c->L + kk] % m, m);
            int in_digit = (u >= lo && u < hi);
            for (int kk = 0; kk < N; kk++) {
                u64 v = madd(msub(0, t[kk], m), mred_i64(e[kk], m), m);
                if (in_digit) v = madd(v, mmul(Pm, target[(size_t)gm * N + kk], m), m);
                bj[kk] = v;
            }
            free(sr); free(t);
        }
    }
    free(s); free(e);
}

/* residues of s^2 and of s(X^g) over all L+K moduli ([L+K][N]) */
void or_sk_square(const void *ctx, u64 *out)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N, nm = c->L + c->K;
    i64 *s = (i64 *)malloc(sizeof(i64) * N);
    or_keygen_sk(ctx, s);
    OR_PARALLEL_FOR
    for (int u = 0; u < nm; u++) {
        u64 *sr = (u64 *)malloc(sizeof(u64) * N);
        for (int k = 0; k < N; k++) sr[k] = mred_i64(s[k], c->mod[u]);
        or_polymul(sr, sr, out + (size_t)u * N, c->logN, c->mod[u], c->psi[u]);
        free(sr);
    }
    free(s);
}

/* automorphism X -> X^g on one residue polynomial: coefficient i moves to
 * g*i mod 2N, negated when that exponent is >= N (X^N = -1) */
void or_automorphism(const u64 *a, u64 *out, int logN, u64 g, u64 m)
{
    const u64 N = (u64)1 << logN, twoN = N << 1;
    for (u64 i = 0; i < N; i++) {
        u64 e = (g * i) % twoN;
        if (e < N) out[e] = a[i] % m;
        else out[e - N] = msub(0, a[i], m);
    }
}

void or_sk_galois(const void *ctx, u64 g, u64 *out)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N, nm = c->L + c->K;
    i64 *s = (i64 *)malloc(sizeof(i64) * N);
    or_keygen_sk(ctx, s);
    OR_PARALLEL_FOR
    for (int u = 0; u < nm; u++) {
        u64 *sr = (u64 *)malloc(sizeof(u64) * N);
        for (int k = 0; k < N; k++) sr[k] = mred_i64(s[k], c->mod[u]);
        or_automorphism(sr, out + (size_t)u * N, c->logN, g, c->mod[u]);
        free(sr);
    }
    free(s);
}

/* ------------------------------------------------------------------ */
/* encryption / decryption (paper: Encrypt, Decrypt)                    */
/* ------------------------------------------------------------------ */
/* ct = (v b + m + e0, v a + e1) mod q_i for i < l; pk_b, pk_a are [L][N];
 * m is [l][N]; ct is [2][l][N] */
void or_encrypt(const void *ctx, const u64 *m, int l, u64 enc_id, const u64 *pk_b,
                const u64 *pk_a, u64 *ct)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N;
    i64 *v = (i64 *)malloc(sizeof(i64) * N), *e0 = (i64 *)malloc(sizeof(i64) * N),
        *e1 = (i64 *)malloc(sizeof(i64) * N);
    or_sample_ternary(c->seed, OBJ_ENC_V(enc_id), c->logN, v);
    or_sample_cbd(c->seed, OBJ_ENC_E0(enc_id), c->logN, e0);
    or_sample_cbd(c->seed, OBJ_ENC_E1(enc_id), c->logN, e1);
    OR_PARALLEL_FOR
    for (int i = 0; i < l; i++) {
        u64 q = c->mod[i];
        u64 *vr = (u64 *)malloc(sizeof(u64) * N), *t = (u64 *)malloc(sizeof(u64) * N);
        for (int k = 0; k < N; k++) vr[k] = mred_i64(v[k], q);
        u64 *c0 = ct + (size_t)i * N, *c1 = ct + ((size_t)l + i) * N;
        or_polymul(vr, pk_b + (size_t)i * N, t, c->logN, q, c->psi[i]);
        for (int k = 0; k < N; k++)
            c0[k] = madd(madd(t[k], m[(size_t)i * N + k], q), mred_i64(e0[k], q), q);
        or_polymul(vr, pk_a + (size_t)i * N, t, c->logN, q, c->psi[i]);
        for (int k = 0; k < N; k++) c1[k] = madd(t[k], mred_i64(e1[k], q), q);
        free(vr); free(t);
    }
    free(v); free(e0); free(e1);
}

/* m = c0 + c1 s mod q_i; ct is [2][l][N], m is [l][N] */
void or_decrypt(const void *ctx, const u64 *ct, int l, u64 *m)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N;
    i64 *s = (i64 *)malloc(sizeof(i64) * N);
    or_keygen_sk(ctx, s);
    OR_PARALLEL_FOR
    for (int i = 0; i < l; i++) {
        u64 q = c->mod[i];
        u64 *sr = (u64 *)malloc(sizeof(u64) * N), *t = (u64 *)malloc(sizeof(u64) * N);
        for (int k = 0; k < N; k++) sr[k] = mred_i64(s[k], q);
        or_polymul(ct + ((size_t)l + i) * N, sr, t, c->logN, q, c->psi[i]);
        for (int k = 0; k < N; k++) m[(size_t)i * N + k] = madd(ct[(size_t)i * N + k], t[k], q);
        free(sr); free(t);
    }
    free(s);
}

/* ------------------------------------------------------------------ */
/* ring operations on q-limb polynomials ([npoly][l][N])                */
/* ------------------------------------------------------------------ */
/* out[p][i] = a[p][i] * b[0][i] (product of every poly of a with one
 * plaintext polynomial b) */
void or_mul_plain(const void *ctx, const u64 *a, int npoly, const u64 *b, int l, u64 *out)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N;
    OR_PARALLEL_FOR_COLLAPSE2
    for (int p = 0; p < npoly; p++)
        for (int i = 0; i < l; i++)
            or_polymul(a + ((size_t)p * l + i) * N, b + (size_t)i * N,
                       out + ((size_t)p * l + i) * N, c->logN, c->mod[i], c->psi[i]);
}

/* tensor of two ciphertexts: (a0 b0, a0 b1 + a1 b0, a1 b1); out is [3][l][N] */
void or_tensor(const void *ctx, const u64 *a, const u64 *b, int l, u64 *out)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N;
    OR_PARALLEL_FOR
    for (int i = 0; i < l; i++) {
        u64 q = c->mod[i];
        u64 *t = (u64 *)malloc(sizeof(u64) * N);
        const u64 *a0 = a + (size_t)i * N, *a1 = a + ((size_t)l + i) * N;
        const u64 *b0 = b + (size_t)i * N, *b1 = b + ((size_t)l + i) * N;
        u64 *d0 = out + (size_t)i * N, *d1 = out + ((size_t)l + i) * N,
            *d2 = out + ((size_t)2 * l + i) * N;
        or_polymul(a0, b0, d0, c->logN, q, c->psi[i]);
        or_polymul(a1, b1, d2, c->logN, q, c->psi[i]);
        or_polymul(a0, b1, d1, c->logN, q, c->psi[i]);
        or_polymul(a1, b0, t, c->logN, q, c->psi[i]);
        for (int k = 0; k < N; k++) d1[k] = madd(d1[k], t[k], q);
        free(t);
    }
}

/* rescale (paper: Rescale) in RNS form: drops q_{l-1}.  For the CRT integer
 * C of each coefficient the result is floor((C + h)/q_{l-1}) with
 * h = floor(q_{l-1}/2), computed limb-wise as (c_i - [(c_{l-1}+h) mod q_{l-1}
 * - h]_{q_i}) * q_{l-1}^{-1} mod q_i.  in [npoly][l][N] -> out [npoly][l-1][N] */
void or_rescale(const void *ctx, const u64 *in, int npoly, int l, u64 *out)
{
    const or_ctx *c = (const or_ctx *)ctx;
    const int N = c->N;
    const u64 ql = c->mod[l - 1], h = ql / 2;
    OR_PARALLEL_FOR_COLLAPSE2
    for (int p = 0; p < npoly; p++) {
        for (int i = 0; i < l - 1; i++) {
            const u64 *last = in + ((size_t)p * l + (l - 1)) * N;
            u64 q = c->mod[i];
            u64 qlinv = minv(ql % q, q);
            const u64 *ci = in + ((size_t)p * l + i) * N;
            u64 *oi = out + ((size_t)p * (l - 1) + i) * N;
            for (int k = 0; k < N; k++) {
                u64 r = (u64)(((u128)last[k] + h) % ql);
                /* v = r - h as a signed value, reduced mod q */
                u64 v = (r >= h) ? (r - h) % q : msub(0, (h - r) % q, q);
                oi[k] = mmul(msub(ci[k], v, q), qlinv, q);
            }
        }
    }
}

/* Hybrid key switching (in the form of the full-RNS CKKS literature; the paper
 * only names the relinearisation and rotation keys):
 *   digits j: q-limbs [j alpha, min(j alpha + alpha, l))
 *   ModUp_j : y_i = [x_i (Q_j/q_i)^-1]_{q_i};  ext_t = sum_i y_i (Q_j/q_i) mod t
 *   inner   : acc_t = sum_j ext_{j,t} * ksk_j,t (negacyclic products)
 *   ModDown : z_k = [acc_{p_k} (P/p_k)^-1]_{p_k};  conv_i = sum_k z_k (P/p_k) mod q_i;
 *             out_i = (acc_i - conv_i) P^-1 mod q_i
 * with P the product of the K_l special primes of the level. */
/* Hybrid key switch of x (coefficient domain, l limbs) with key families of
 * K_l = or_ks_special(l) special primes (built by or_keygen_ksk with that k
 * and key_lmax >= l): ModUp per digit, inner product, ModDown by P_{K_l}.
 *
 * With ngal > 0 this is the hoisted sum over Galois elements gal[0..ngal):
 * the ModUp digits are computed once, each element's automorphism is applied
 * to them (limb by limb, modulo that limb's modulus), their inner products
 * with the element's key (ksk holds ngal families back to back) are summed in
 * the extended basis, and one ModDown follows.  ngal = 0 is the plain switch
 * of x with the one key in ksk. */
static void keyswitch_sum(const or_ctx *c, const u64 *x, int l, int ngal, const u64 *gal,
                          const u64 *ksk, int key_lmax, const u64 *fuse, u64 *out);

void or_keyswitch(const void *ctx, const u64 *x, int l, const u64 *ksk, int key_lmax, u64 *out)
{
    keyswitch_sum((const or_ctx *)ctx, x, l, 0, NULL, ksk, key_lmax, NULL, out);
}

void or_keyswitch_hoisted(const void *ctx, const u64 *x, int l, int ngal, const u64 *gal,
                          const u64 *ksk, int key_lmax, u64 *out)
{
    keyswitch_sum((const or_ctx *)ctx, x, l, ngal, gal, ksk, key_lmax, NULL, out);
}

/* Relinearisation fused with the rescale that follows it (A tensor (d0, d1,
 * d2) at level l, coefficient domain [3][l][N] -> [2][l-1][N]): the key
 * product acc of d2 is not divided by P and then the sum by q_{l-1}; instead
 * y = acc + P (d0, d1) is divided once by P' = P q_{l-1}, rounding to nearest:
 *   B' = {p_0..p_{K-1}, q_{l-1}},  h = (P' - 1) / 2,
 *   z_j   = [(y_j + h) (P'/m_j)^-1]_{m_j}           for m_j in B'
 *   conv_i = sum_j z_j (P'/m_j) mod q_i             for i < l - 1
 *   out_i = (y_i + h - conv_i) P'^-1 mod q_i. */
void or_relin_rescale(const void *ctx, const u64 *t3, int l, const u64 *ksk, int key_lmax,
                      u64 *out)
{
    keyswitch_sum((const or_ctx *)ctx, t3 + (size_t)2 * l * ((const or_ctx *)ctx)->N, l, 0,
                  NULL, ksk, key_lmax, t3, out);
}

static void keyswitch_sum(const or_ctx *c, const u64 *x, int l, int ngal, const u64 *gal,
                          const u64 *ksk, int key_lmax, const u64 *fuse, u64 *out)
{
    const int N = c->N, L = c->L, K = c->ks_k[l], nm = key_lmax + K, ne = l + K;
    const int beta = (l + c->alpha - 1) / c->alpha;
    u64 emod[OR_MAXMOD];
    int ekey[OR_MAXMOD]; /* row of the key for extended limb u */
    for (int u = 0; u < ne; u++) {
        emod[u] = u < l ? c->mod[u] : c->mod[L + (u - l)];
        ekey[u] = u < l ? u : key_lmax + (u - l);
    }
    u64 *ext = (u64 *)malloc(sizeof(u64) * (size_t)beta * ne * N);
    u64 *acc = (u64 *)calloc((size_t)2 * ne * N, sizeof(u64));
    /* ModUp, digit by digit */
    for (int j = 0; j < beta; j++) {
        int lo = j * c->alpha, hi = lo + c->alpha < l ? lo + c->alpha : l;
        u64 *ej = ext + (size_t)j * ne * N;
        u64 hinv[OR_MAXMOD];            /* (Q_j/q_i)^-1 mod q_i        */
        u64 hmod[OR_MAXMOD][OR_MAXMOD]; /* (Q_j/q_i) mod emod[u]        */
        for (int i = lo; i < hi; i++) {
            u64 qh = 1;
            for (int i2 = lo; i2 < hi; i2++) if (i2 != i) qh = mmul(qh, c->mod[i2] % c->mod[i], c->mod[i]);
            hinv[i - lo] = minv(qh, c->mod[i]);
            for (int u = 0; u < ne; u++) {
                u64 m = emod[u], h = 1;
                for (int i2 = lo; i2 < hi; i2++) if (i2 != i) h = mmul(h, c->mod[i2] % m, m);
                hmod[i - lo][u] = h;
            }
        }
        OR_PARALLEL_FOR
        for (int k = 0; k < N; k++) {
            u64 y[OR_MAXMOD];
            for (int i = lo; i < hi; i++) y[i - lo] = mmul(x[(size_t)i * N + k], hinv[i - lo], c->mod[i]);
            for (int u = 0; u < ne; u++) {
                if (u >= lo && u < hi) { ej[(size_t)u * N + k] = x[(size_t)u * N + k]; continue; }
                u64 m = emod[u], s = 0;
                for (int i = lo; i < hi; i++) s = madd(s, mmul(y[i - lo] % m, hmod[i - lo][u], m), m);
                ej[(size_t)u * N + k] = s;
            }
        }
    }
    /* inner product with the key (or the sum over the automorphisms' keys) */
    const int dk = (key_lmax + c->alpha - 1) / c->alpha;
    const size_t fam_words = (size_t)dk * 2 * nm * N;
    for (int gi = 0; gi < (ngal > 0 ? ngal : 1); gi++) {
        const u64 *key = ksk + (size_t)gi * fam_words;
        OR_PARALLEL_FOR_COLLAPSE2
        for (int pz = 0; pz < 2; pz++)
            for (int u = 0; u < ne; u++) {
                u64 *t = (u64 *)malloc(sizeof(u64) * N), *sg = (u64 *)malloc(sizeof(u64) * N);
                u64 m = emod[u];
                u64 psi = u < l ? c->psi[u] : c->psi[L + (u - l)];
                u64 *a = acc + ((size_t)pz * ne + u) * N;
                for (int j = 0; j < beta; j++) {
                    const u64 *kj = key + (((size_t)j * 2 + pz) * nm + ekey[u]) * N;
                    const u64 *ej = ext + ((size_t)j * ne + u) * N;
                    if (ngal > 0) {
                        or_automorphism(ej, sg, c->logN, gal[gi], m);
                        ej = sg;
                    }
                    or_polymul(ej, kj, t, c->logN, m, psi);
                    for (int k = 0; k < N; k++) a[k] = madd(a[k], t[k], m);
                }
                free(t); free(sg);
            }
    }
    if (fuse) {
        /* ModDown fused with the rescale: divide y = acc + P (d0, d1) by
         * P' = P q_{l-1} through B' = {p_0..p_{K-1}, q_{l-1}} */
        const int nb = K + 1, lo = l - 1;
        u64 bm[OR_MAXMOD];
        int brow[OR_MAXMOD];
        for (int kk = 0; kk < K; kk++) { bm[kk] = c->mod[L + kk]; brow[kk] = l + kk; }
        bm[K] = c->mod[l - 1];
        brow[K] = l - 1;
        u64 Pq[OR_MAXMOD];                /* P mod q_i, i < l         */
        for (int i = 0; i < l; i++) {
            Pq[i] = 1;
            for (int kk = 0; kk < K; kk++) Pq[i] = mmul(Pq[i], c->mod[L + kk] % c->mod[i], c->mod[i]);
        }
        u64 bhinv[OR_MAXMOD], hb[OR_MAXMOD];  /* (P'/m_j)^-1 mod m_j, h mod m_j */
        u64 bh[OR_MAXMOD][OR_MAXMOD];         /* (P'/m_j) mod q_i          */
        for (int j = 0; j < nb; j++) {
            u64 m = bm[j], r = 1;
            for (int j2 = 0; j2 < nb; j2++) if (j2 != j) r = mmul(r, bm[j2] % m, m);
            bhinv[j] = minv(r, m);
            hb[j] = (m - 1) / 2;          /* P' = 0 mod m: h = -1/2 mod m */
            for (int i = 0; i < lo; i++) {
                u64 q = c->mod[i], v = 1;
                for (int j2 = 0; j2 < nb; j2++) if (j2 != j) v = mmul(v, bm[j2] % q, q);
                bh[j][i] = v;
            }
        }
        u64 ppinv[OR_MAXMOD], hq[OR_MAXMOD];  /* P'^-1 mod q_i, h mod q_i */
        for (int i = 0; i < lo; i++) {
            u64 q = c->mod[i], Pp = 1;
            for (int j = 0; j < nb; j++) Pp = mmul(Pp, bm[j] % q, q);
            ppinv[i] = minv(Pp, q);
            hq[i] = mmul(msub(Pp, 1, q), (q + 1) / 2, q);
        }
        for (int pz = 0; pz < 2; pz++) {
            const u64 *a = acc + (size_t)pz * ne * N, *d = fuse + (size_t)pz * l * N;
            OR_PARALLEL_FOR
            for (int k = 0; k < N; k++) {
                u64 z[OR_MAXMOD];
                for (int j = 0; j < nb; j++) {
                    u64 m = bm[j], y = a[(size_t)brow[j] * N + k];
                    if (j == K) y = madd(y, mmul(Pq[l - 1], d[(size_t)(l - 1) * N + k], m), m);
                    z[j] = mmul(madd(y, hb[j], m), bhinv[j], m);
                }
                for (int i = 0; i < lo; i++) {
                    u64 q = c->mod[i], conv = 0;
                    for (int j = 0; j < nb; j++) conv = madd(conv, mmul(z[j] % q, bh[j][i], q), q);
                    u64 y = madd(a[(size_t)i * N + k], mmul(Pq[i], d[(size_t)i * N + k], q), q);
                    out[((size_t)pz * lo + i) * N + k] =
                        mmul(msub(madd(y, hq[i], q), conv, q), ppinv[i], q);
                }
            }
        }
        free(ext); free(acc);
        return;
    }
    /* ModDown */
    u64 phinv[OR_MAXMOD];           /* (P/p_k)^-1 mod p_k */
    u64 phmod[OR_MAXMOD][OR_MAXMOD]; /* (P/p_k) mod q_i    */
    u64 pinv[OR_MAXMOD];            /* P^-1 mod q_i       */
    for (int kk = 0; kk < K; kk++) {
        u64 pk = c->mod[L + kk], ph = 1;
        for (int k2 = 0; k2 < K; k2++) if (k2 != kk) ph = mmul(ph, c->mod[L + k2] % pk, pk);
        phinv[kk] = minv(ph, pk);
        for (int i = 0; i < l; i++) {
            u64 q = c->mod[i], h = 1;
            for (int k2 = 0; k2 < K; k2++) if (k2 != kk) h = mmul(h, c->mod[L + k2] % q, q);
            phmod[kk][i] = h;
        }
    }
    for (int i = 0; i < l; i++) {
        u64 q = c->mod[i], P = 1;
        for (int kk = 0; kk < K; kk++) P = mmul(P, c->mod[L + kk] % q, q);
        pinv[i] = minv(P, q);
    }
    for (int pz = 0; pz < 2; pz++) {
        const u64 *a = acc + (size_t)pz * ne * N;
        OR_PARALLEL_FOR
        for (int k = 0; k < N; k++) {
            u64 z[OR_MAXMOD];
            for (int kk = 0; kk < K; kk++)
                z[kk] = mmul(a[(size_t)(l + kk) * N + k], phinv[kk], c->mod[L + kk]);
            for (int i = 0; i < l; i++) {
                u64 q = c->mod[i], conv = 0;
                for (int kk = 0; kk < K; kk++) conv = madd(conv, mmul(z[kk] % q, phmod[kk][i], q), q);
                out[((size_t)pz * l + i) * N + k] = mmul(msub(a[(size_t)i * N + k], conv, q), pinv[i], q);
            }
        }
    }
    free(ext); free(acc);
}

/* ------------------------------------------------------------------ */
/* encoding (paper: Encode / Decode via the canonical embedding phi)    */
/* ------------------------------------------------------------------ */
/* Twiddles of the encoding procedure, from their definition with the C
 * library's cos/sin:
 *   W[t] = exp(-2 pi i t / M) for t < M/2, angle computed as (t * 2pi) / M
 *   T[k] = exp(-pi i k / N)   for k < M,   angle computed as (k * pi) / N
 * sign = -1 gives these (encoding); sign = +1 their conjugates (decoding). */
static const double OR_PI = 3.14159265358979323846;
void or_fft_twiddles(int logN, int sign, double *W /*[M/2][2]*/, double *T /*[M][2]*/)
{
    const int N = 1 << logN, M = N / 2;
    for (int t = 0; t < M / 2; t++) {
        double ang = ((double)t * (2.0 * OR_PI)) / (double)M;
        W[2 * t] = cos(ang);
        W[2 * t + 1] = (double)sign * sin(ang);
    }
    for (int k = 0; k < M; k++) {
        double ang = ((double)k * OR_PI) / (double)N;
        T[2 * k] = cos(ang);
        T[2 * k + 1] = (double)sign * sin(ang);
    }
}

/* slot j sits at rotation-group index u_j = ((5^j mod 2N) - 1) / 4 */
static void slot_index(int logN, int *u)
{
    const u64 twoN = (u64)2 << logN;
    const int M = 1 << (logN - 1);
    u64 g = 1;
    for (int j = 0; j < M; j++) {
        u[j] = (int)((g - 1) / 4);
        g = (g * 5) % twoN;
    }
}

static int bitrev(int x, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; b++) r |= ((x >> b) & 1) << (bits - 1 - b);
    return r;
}

/* Encoding procedure, exact fixed-point integer arithmetic:
 *   e  = smallest integer >= 0 with 2^e >= max_j max(|Re z_j|, |Im z_j|), capped at 40
 *   F  = 61 - log2(M) - e fractional bits;  Z_j = (llrint(Re z_j 2^F), llrint(Im z_j 2^F))
 *   twiddles Wq[t] = llrint(W[t] 2^62), Tq[k] = llrint(T[k] 2^62) (W, T as above)
 *   complex product a * w = (ar wr - ai wi, ar wi + ai wr) computed exactly on
 *   128 bits, each part rounded to (v + 2^61) >> 62 (arithmetic shift)
 *   G[bitrev(u_j)] = Z_j;  for len = 2, 4, ..., M, block b, jj < len/2:
 *       y = G[b+jj+len/2] * Wq[jj (M/len)];  G[b+jj] = x + y;  G[b+jj+len/2] = x - y
 *   c_k = G[k] * Tq[k];  f = scale / 2^(log2 M + F) (a double, exact power-of-two
 *   scaling); coefficient k = llrint((double)Re c_k * f), k + M = llrint((double)Im c_k * f)
 * This inverts the canonical embedding m(zeta^(5^j)) = scale * z_j with
 * zeta = exp(i pi / N).  Every value stays below 2^61.5 (inputs <= 2^(61-logM)
 * grow at most 2^logM * sqrt 2); |z| <= 2^40 is required.  The result differs
 * from the exact embedding's rounding by at most about scale * 2^-F.
 * z is [M][2] (re, im); out is [N] signed integers. */
typedef __int128 i128;
static i64 rshift62(i128 v) { return (i64)((v + ((i128)1 << 61)) >> 62); }
static void cmul_fx(i64 ar, i64 ai, i64 wr, i64 wi, i64 *rr, i64 *ri)
{
    *rr = rshift62((i128)ar * wr - (i128)ai * wi);
    *ri = rshift62((i128)ar * wi + (i128)ai * wr);
}

int or_encode_exponent(const double *z, int M)
{
    double mx = 0.0;
    for (int j = 0; j < 2 * M; j++) {
        double a = fabs(z[j]);
        if (a > mx) mx = a;
    }
    int e = 0;
    while (e < 40 && ldexp(1.0, e) < mx) e++;
    return e;
}

void or_encode(int logN, const double *z, double scale, i64 *out)
{
    const int N = 1 << logN, M = N / 2, logM = logN - 1;
    double *W = (double *)malloc(sizeof(double) * M);
    double *T = (double *)malloc(sizeof(double) * 2 * M);
    i64 *Wq = (i64 *)malloc(sizeof(i64) * M);
    i64 *Tq = (i64 *)malloc(sizeof(i64) * 2 * M);
    i64 *G = (i64 *)malloc(sizeof(i64) * 2 * M);
    int *u = (int *)malloc(sizeof(int) * M);
    or_fft_twiddles(logN, -1, W, T);
    for (int t = 0; t < M; t++) Wq[t] = llrint(ldexp(W[t], 62));
    for (int k = 0; k < 2 * M; k++) Tq[k] = llrint(ldexp(T[k], 62));
    slot_index(logN, u);
    const int e = or_encode_exponent(z, M);
    const int F = 61 - logM - e;
    for (int j = 0; j < M; j++) {
        int p = bitrev(u[j], logM);
        G[2 * p] = llrint(ldexp(z[2 * j], F));
        G[2 * p + 1] = llrint(ldexp(z[2 * j + 1], F));
    }
    for (int len = 2; len <= M; len <<= 1) {
        int half = len / 2, stride = M / len;
        for (int b = 0; b < M; b += len)
            for (int jj = 0; jj < half; jj++) {
                i64 *x = G + 2 * (b + jj), *y = G + 2 * (b + jj + half);
                i64 tr, ti;
                cmul_fx(y[0], y[1], Wq[2 * (jj * stride)], Wq[2 * (jj * stride) + 1], &tr, &ti);
                i64 xr = x[0], xi = x[1];
                x[0] = xr + tr; x[1] = xi + ti;
                y[0] = xr - tr; y[1] = xi - ti;
            }
    }
    const double f = ldexp(scale, -(logM + F));
    for (int k = 0; k < M; k++) {
        i64 cr, ci;
        cmul_fx(G[2 * k], G[2 * k + 1], Tq[2 * k], Tq[2 * k + 1], &cr, &ci);
        out[k] = llrint((double)cr * f);
        out[k + M] = llrint((double)ci * f);
    }
    free(W); free(T); free(Wq); free(Tq); free(G); free(u);
}

/* signed coefficients -> residues over q_0..q_{l-1} ([l][N]) */
void or_to_rns(const void *ctx, const i64 *v, int l, u64 *out)
{
    const or_ctx *c = (const or_ctx *)ctx;
    signed_to_rns(c, v, c->mod, l, out);
}

/* residues over moduli mods[0..n) for arbitrary moduli (used for keys) */
void or_to_rns_mods(int logN, const i64 *v, const u64 *mods, int n, u64 *out)
{
    const int N = 1 << logN;
    for (int u = 0; u < n; u++)
        for (int k = 0; k < N; k++) out[(size_t)u * N + k] = mred_i64(v[k], mods[u]);
}
