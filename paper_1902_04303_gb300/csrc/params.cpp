// params.cpp -- host-side parameter generation of the gwhe library: the RNS
// basis, primitive roots, Shoup/Barrett constants and the twiddles of the
// encoding procedure.  Compiled with -ffp-contract=off: the twiddles are
// defined as separately rounded IEEE operations.
#include <cmath>
#include <cstdint>
#include <vector>

#include "core.cuh"

namespace gwhe {

u64 host_mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * (u128)b) % m); }

u64 host_powmod(u64 a, u64 e, u64 m) {
  u64 result = 1 % m, base = a % m;
  for (; e; e >>= 1) {
    if (e & 1) result = host_mulmod(result, base, m);
    base = host_mulmod(base, base, m);
  }
  return result;
}

u64 host_inv(u64 a, u64 m) { return host_powmod(a % m, m - 2, m); }  // m prime

// Miller-Rabin with the twelve smallest prime bases: deterministic below 2^64.
static bool is_prime64(u64 n) {
  static const u64 witnesses[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 w : witnesses)
    if (n % w == 0) return n == w;
  int s = 0;
  u64 odd = n - 1;
  while (!(odd & 1)) {
    odd >>= 1;
    ++s;
  }
  for (u64 w : witnesses) {
    u64 x = host_powmod(w, odd, n);
    if (x == 1 || x == n - 1) continue;
    bool witness_composite = true;
    for (int r = 1; r < s && witness_composite; ++r) {
      x = host_mulmod(x, x, n);
      if (x == n - 1) witness_composite = false;
    }
    if (witness_composite) return false;
  }
  return true;
}

// RNS basis (see the library header for the rule): base prime = largest
// prime < 2^q0_bits congruent to 1 mod 2N; scale primes = the candidates
// nearest 2^scale_bits taken alternately below and above; special primes = the
// next largest below 2^sp_bits.  All distinct.
int gen_primes(int logN, int L, int q0_bits, int scale_bits, int K, int sp_bits, u64* q, u64* p) {
  if (L < 1 || K < 1 || L + K > kMaxMod) return ST_EINVAL;
  if (q0_bits > 60 || sp_bits > 60 || scale_bits > 60 || logN < 2 || logN > 17) return ST_EINVAL;
  const u64 twoN = (u64)1 << (logN + 1);
  std::vector<u64> taken;
  auto is_taken = [&](u64 v) {
    for (u64 t : taken)
      if (t == v) return true;
    return false;
  };
  auto next_down = [&](u64& cand) -> bool {  // first usable candidate <= cand
    while (cand > twoN && (!is_prime64(cand) || is_taken(cand))) cand -= twoN;
    return cand > twoN;
  };
  u64 cand = ((u64)1 << q0_bits) - twoN + 1;
  if (!next_down(cand)) return ST_EINVAL;
  q[0] = cand;
  taken.push_back(cand);
  u64 lower = ((u64)1 << scale_bits) - twoN + 1;
  u64 upper = ((u64)1 << scale_bits) + 1;
  for (int i = 1; i < L; ++i) {
    if (i & 1) {
      if (!next_down(lower)) return ST_EINVAL;
      q[i] = lower;
      lower -= twoN;
    } else {
      while (!is_prime64(upper) || is_taken(upper)) upper += twoN;
      q[i] = upper;
      upper += twoN;
    }
    taken.push_back(q[i]);
  }
  u64 sp = ((u64)1 << sp_bits) - twoN + 1;
  for (int k = 0; k < K; ++k) {
    if (!next_down(sp)) return ST_EINVAL;
    p[k] = sp;
    taken.push_back(sp);
    sp -= twoN;
  }
  return ST_OK;
}

// A primitive 2N-th root of unity mod q (psi^N = -1).  Any such root works:
// the library compares and exchanges polynomials in the coefficient domain.
u64 find_psi(u64 q, int logN) {
  const u64 N = (u64)1 << logN;
  for (u64 g = 2; g < 1000000; ++g) {
    u64 r = host_powmod(g, (q - 1) / (2 * N), q);
    if (host_powmod(r, N, q) == q - 1) return r;
  }
  throw Error(ST_EINVAL, "no primitive 2N-th root found");
}

u64 shoup_companion(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

DevMod make_devmod(u64 q) {
  DevMod m;
  m.q = q;
  m.twoq = 2 * q;
  m.R = (u64)(((u128)1 << 64) % q);
  m.Rsh = shoup_companion(m.R, q);
  m.mu = (u64)(((u128)1 << 64) / q);
  return m;
}

int bitrev_host(int x, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b)
    if (x & (1 << b)) r |= 1 << (bits - 1 - b);
  return r;
}

// Twiddles of the encoding procedure, from the definition:
//   W[t] = exp(sign 2 pi i t / M), angle (t * 2pi) / M, for t < M/2
//   T[k] = exp(sign pi i k / N),   angle (k * pi) / N,   for k < M
// with the C library's cos and sin (sign = -1 encodes, +1 decodes).
void fft_twiddles(int logN, int sign, double* W, double* T) {
  const double kPi = 3.14159265358979323846;
  const int N = 1 << logN, M = N >> 1;
  for (int t = 0; t < M / 2; ++t) {
    const double angle = ((double)t * (2.0 * kPi)) / (double)M;
    W[2 * t] = std::cos(angle);
    W[2 * t + 1] = (double)sign * std::sin(angle);
  }
  for (int k = 0; k < M; ++k) {
    const double angle = ((double)k * kPi) / (double)N;
    T[2 * k] = std::cos(angle);
    T[2 * k + 1] = (double)sign * std::sin(angle);
  }
}

}  // namespace gwhe
