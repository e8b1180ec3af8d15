// noalloc.cu -- a key switch that allocates no device memory.
//
// Some callers cannot let the library call cudaMalloc: a serving process whose
// device memory is reserved up front by its own pool (so any further
// allocation fails or fragments it), or a latency-bound request path where an
// allocator call may block on or synchronise the device.  For them
// gwhe_keyswitch_noalloc runs the same hybrid key switch as the rest of the
// library, with every temporary (the coefficient copy of the input, the
// ModUp digits, the key products, the ModDown conversion) carved out of one
// file-scope device array of fixed size instead of the memory pool.
//
// The array is a module-level __device__ object: every GPU that loads the
// library holds it until the process exits.  Host code cannot use its name as
// a device address; its address on a device is looked up with
// cudaGetSymbolAddress, with that device current, when a context is created
// there (ctx_create), which also loads this file's module and commits the
// array's memory, so the entry point's own calls reserve nothing.
#include "capi_types.cuh"

using namespace gwhe;

namespace {

// 32 MiB of scratch (2^22 words).  A key switch at level l needs
// (3 l + (beta + 2) (l + K_l)) N words with beta = ceil(l / alpha) digits and
// K_l the special primes that level uses.
constexpr size_t kScratchWords = (size_t)1 << 22;
static __device__ __align__(256) u64 g_ks_scratch[kScratchWords];

}  // namespace

namespace gwhe {

u64* noalloc_scratch_lookup() {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_ks_scratch);
  if (e != cudaSuccess)
    throw Error(ST_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  return (u64*)p;
}

}  // namespace gwhe

extern "C" int gwhe_keyswitch_noalloc(gwhe_ctx* ctx, const uint64_t* x_ntt, int l,
                                      uint32_t key_id, uint64_t* out_ntt) {
  Context* c = ctx ? ctx->c : nullptr;
  if (!c) return GWHE_EINVAL;
  try {
    if (!x_ntt || !out_ntt || l < 1 || l > c->P.L)
      throw Error(ST_EINVAL, "keyswitch_noalloc: bad arguments");
    const Ksk& fam = key_family(c, key_id, l);
    const size_t N = c->N;
    const int K = fam.k, L = c->P.L, ne = l + K;
    const int beta = (l + c->alpha - 1) / c->alpha;
    const size_t need = ((size_t)3 * l + (size_t)(beta + 2) * ne) * N;
    if (need > kScratchWords)
      throw Error(ST_EINVAL, "keyswitch_noalloc: level " + std::to_string(l) + " needs " +
                                 std::to_string(need) + " scratch words, the static array holds " +
                                 std::to_string(kScratchWords));
    // the array of the context's device (its keys and tables live there too)
    require_device(c);
    u64* base = c->noalloc_scratch;
    if (!base) throw Error(ST_ECUDA, "keyswitch_noalloc: scratch array not resolved");
    // carve the scratch: nothing in it needs to start at zero (every region
    // is fully written before it is read)
    u64* xc = base;                          // [l][N]  input, coefficient domain
    u64* ext = xc + (size_t)l * N;           // [beta][ne][N] ModUp digits
    u64* acc = ext + (size_t)beta * ne * N;  // [2][ne][N] key products
    u64* conv = acc + (size_t)2 * ne * N;    // [2][l][N] ModDown conversion
    ++c->ks_count;
    ++c->ks_by_level[l];
    GWHE_CUDA(cudaMemcpyAsync(xc, x_ntt, sizeof(u64) * l * N, cudaMemcpyDeviceToDevice, c->stream));
    ntt_inverse(c, xc, rows_q(1, l, l));
    modup_convert_set(c, xc, l, ext, 1);
    for (int j = 0; j < beta; ++j) {
      const ConvTable& t = c->modup.at({l, j});
      RowMap rm;
      rm.npoly = 1;
      rm.nl = t.n_out;
      rm.poly_stride = ne;
      for (int o = 0; o < t.n_out; ++o) {
        rm.off[o] = t.out_limb[o];
        rm.pidx[o] = t.out_pidx[o];
      }
      ntt_forward(c, ext + (size_t)j * ne * N, rm);
    }
    ks_inner_set(c, x_ntt, 0, l, ext, fam, acc, 1);
    RowMap rk;
    rk.npoly = 2;
    rk.nl = K;
    rk.poly_stride = ne;
    for (int k = 0; k < K; ++k) {
      rk.off[k] = (uint16_t)(l + k);
      rk.pidx[k] = (uint8_t)(L + k);
    }
    ntt_inverse(c, acc, rk);
    moddown_convert_set(c, acc, l, K, conv, 1);
    ntt_forward(c, conv, rows_q(2, l, l));
    moddown_combine_set(c, acc, conv, l, K, 1, out_ntt, out_ntt + (size_t)l * N, 0, nullptr,
                        nullptr, 0, 0);
    return GWHE_OK;
  } catch (const Error& e) {
    c->last_error = e.what();
    return e.code;
  } catch (const std::exception& e) {
    c->last_error = e.what();
    return GWHE_EINVAL;
  }
}
