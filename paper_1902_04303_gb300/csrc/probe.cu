// probe.cu -- the arithmetic ceiling of the NTT butterfly on this GPU.
//
// The NTT is bound by 64-bit modular integer arithmetic, not by memory: the
// GPU has no 64-bit integer multiplier, so each Shoup product is a sequence of
// 32-bit multiply-adds.  This kernel runs the transform's own Cooley-Tukey
// butterfly (ct_bfly) on residues held in registers, with no memory traffic
// in the loop, across every SM.  Its rate is the ceiling that a butterfly
// kernel cannot pass; the NTT's achieved butterfly rate is reported against it.
#include <vector>

#include "capi_types.cuh"

using namespace gwhe;

namespace {

// rounds x (4 radix-2 stages over 16 registers = 32 butterflies) per thread
__global__ void __launch_bounds__(256) k_bfly_probe(u64* __restrict__ out, u64 q, const u64* tw,
                                                    int rounds) {
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 q4 = 4 * q, nq = 0 - q;
  u64 w[4], wsh[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    w[s] = tw[2 * s];
    wsh[s] = tw[2 * s + 1];
  }
  u64 x[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) x[m] = (gid * 16 + m) % q;
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int st = 8 >> s;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        if (m & st) continue;
        ct_bfly(x[m], x[m + st], w[s], wsh[s], q4, nq);
      }
    }
  }
  u64 acc = 0;
#pragma unroll
  for (int m = 0; m < 16; ++m) acc ^= x[m];
  out[gid] = acc;
}

}  // namespace

extern "C" int gwhe_probe_butterflies(gwhe_ctx* ctx, int rounds, double* per_s, double* ms) {
  Context* c = ctx ? ctx->c : nullptr;
  if (!c || rounds < 1 || !per_s) return GWHE_EINVAL;
  try {
    int dev = 0, sms = 0;
    GWHE_CUDA(cudaGetDevice(&dev));
    GWHE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int ctas = sms * 8;
    const size_t threads = (size_t)ctas * 256;
    const int u = 0;  // the first q prime and its twiddles psi^brv(1..4)
    std::vector<u64> tw(8);  // 4 (twiddle, Shoup companion) pairs
    GWHE_CUDA(cudaMemcpy(tw.data(), c->d_psi + ((size_t)u << c->logN) + 1, sizeof(ulonglong2) * 4,
                         cudaMemcpyDeviceToHost));
    Tmp out(c, sizeof(u64) * threads), dtw(c, sizeof(u64) * 8);
    GWHE_CUDA(cudaMemcpyAsync(dtw.p, tw.data(), sizeof(u64) * 8, cudaMemcpyHostToDevice, c->stream));
    cudaEvent_t e0, e1;
    GWHE_CUDA(cudaEventCreate(&e0));
    GWHE_CUDA(cudaEventCreate(&e1));
    k_bfly_probe<<<ctas, 256, 0, c->stream>>>(out.u(), c->hmod[u].q, dtw.u(), 1);  // warm-up
    GWHE_CUDA(cudaEventRecord(e0, c->stream));
    k_bfly_probe<<<ctas, 256, 0, c->stream>>>(out.u(), c->hmod[u].q, dtw.u(), rounds);
    GWHE_CUDA(cudaEventRecord(e1, c->stream));
    GWHE_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    GWHE_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GWHE_LAUNCHED(c, 2);
    *per_s = (double)threads * rounds * 32.0 / (t * 1e-3);
    if (ms) *ms = t;
    return GWHE_OK;
  } catch (const Error& e) {
    c->last_error = e.what();
    return e.code;
  }
}
