// bp_sort.cu -- device-wide exclusive scan, stable LSD radix sort of (key, value)
// pairs and per-key range boundaries.  Used to build the (tile, particle) and
// (tile, halo) work lists; everything is deterministic (no order-dependent atomics
// on data: the only atomics are shared-memory histogram counts).
#include "bp_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_PER_THREAD;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix
// and writes the block total to *total.
template <class T>
__device__ T block_excl_scan(T v, T* total) {
  __shared__ T s_w[33];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) s_w[w] = inc;
  __syncthreads();
  if (w == 0) {
    T x = lane < nw ? s_w[lane] : T(0);
    T xi = warp_incl_scan(x);
    if (lane < nw) s_w[lane] = xi - x;
    if (lane == nw - 1) s_w[32] = xi;
  }
  __syncthreads();
  T res = inc - v + s_w[w];
  if (total) *total = s_w[32];
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* in, int64_t n,
                                                              int64_t* bsum) {
  int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  int64_t s = 0;
  for (int k = 0; k < SCAN_PER_THREAD; ++k)
    if (base + k < n) s += in[base + k];
  int64_t tot;
  block_excl_scan<int64_t>(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: in-place exclusive scan of nb block sums; writes the grand total
// to bsum[nb]
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_bsums(int64_t* bsum, int64_t nb) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += SCAN_THREADS) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    int64_t ex = block_excl_scan<int64_t>(v, &tot);
    if (i < nb) bsum[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t* in, int64_t n,
                                                            const int64_t* bsum, int64_t* out) {
  int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  uint32_t v[SCAN_PER_THREAD];
  int64_t s = 0;
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  int64_t ex = block_excl_scan<int64_t>(s, nullptr) + bsum[blockIdx.x];
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = BP_RS_ITEMS;  // items per block (bp_internal.cuh)
constexpr int RS_ROUNDS = RS_ITEMS / RS_THREADS;
static_assert(RS_ROUNDS * RS_THREADS == RS_ITEMS, "radix block");
constexpr int RS_MAXDIG = 256;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t* keys, int64_t n,
                                                        int shift, int nbits, uint32_t* hist,
                                                        int64_t nblocks) {
  __shared__ uint32_t s_h[RS_MAXDIG];
  int ndig = 1 << nbits;
  for (int d = threadIdx.x; d < ndig; d += RS_THREADS) s_h[d] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_ITEMS;
  // all of this thread's keys in flight at once, then the shared-memory counts
  uint32_t kk[RS_ROUNDS];
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
    kk[r] = i < n ? keys[i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&s_h[(kk[r] >> shift) & (ndig - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < ndig; d += RS_THREADS)
    hist[(int64_t)d * nblocks + blockIdx.x] = s_h[d];
}

// Stable scatter of one block of RS_ITEMS items.  Each lane first loads its keys and values
// (RS_SUB of each, all loads in flight together); warp w then ranks the contiguous slice
// [w * RS_ITEMS / 8, (w + 1) * RS_ITEMS / 8) of the block in index order (32 items at a
// time, peers by digit with __match_any_sync, per-warp digit counts in shared memory); the
// block places every item at its digit-sorted position in a shared-memory buffer and
// copies the buffer out, so that the writes of each digit run are contiguous in memory.
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_SUB = RS_ITEMS / RS_WARPS / 32;  // items per lane

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t* kin,
                                                           const uint32_t* vin, uint32_t* kout,
                                                           uint32_t* vout, int64_t n, int shift,
                                                           int nbits, const int64_t* offs,
                                                           int64_t nblocks, int* dbg) {
  __shared__ uint32_t s_cnt[RS_WARPS][RS_MAXDIG];  // per-warp digit counts, then offsets
  __shared__ uint32_t s_tot[RS_MAXDIG];
  __shared__ uint32_t s_start[RS_MAXDIG];          // block-local start of each digit
  __shared__ int64_t s_off[RS_MAXDIG];             // global start of this block's run
  __shared__ uint32_t s_k[RS_ITEMS], s_v[RS_ITEMS];
  const int ndig = 1 << nbits;
  const uint32_t dmask = (uint32_t)(ndig - 1);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int d = tid; d < RS_MAXDIG; d += RS_THREADS) {
    s_off[d] = d < ndig ? offs[(int64_t)d * nblocks + blockIdx.x] : 0;
    for (int q = 0; q < RS_WARPS; ++q) s_cnt[q][d] = 0;
  }
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t bbase = (int64_t)blockIdx.x * RS_ITEMS;
  const int64_t wbase = bbase + (int64_t)w * (RS_ITEMS / RS_WARPS);
  uint32_t kk[RS_SUB], vv[RS_SUB];
#pragma unroll
  for (int j = 0; j < RS_SUB; ++j) {
    const int64_t i = wbase + 32 * j + lane;
    kk[j] = i < n ? kin[i] : 0u;
    vv[j] = i < n ? vin[i] : 0u;
  }
  uint32_t rnk[RS_SUB];
#pragma unroll
  for (int j = 0; j < RS_SUB; ++j) {
    const int64_t i = wbase + 32 * j + lane;
    const bool valid = i < n;
    const uint32_t key = kk[j];
    const uint32_t d = (key >> shift) & dmask;
    const uint32_t tag = valid ? d : (0x80000000u | (uint32_t)lane);
    const uint32_t peers = __match_any_sync(0xffffffffu, tag);
    const uint32_t r = __popc(peers & lt_mask);
    const uint32_t before = valid ? s_cnt[w][d] : 0u;
    __syncwarp();
    if (valid && r == 0) s_cnt[w][d] = before + __popc(peers);
    __syncwarp();
    rnk[j] = before + r;
  }
  __syncthreads();
  // per digit: exclusive offsets of the warps, and the digit's total in the block
  for (int d = tid; d < RS_MAXDIG; d += RS_THREADS) {
    uint32_t run = 0;
    for (int q = 0; q < RS_WARPS; ++q) {
      const uint32_t c = s_cnt[q][d];
      s_cnt[q][d] = run;
      run += c;
    }
    s_tot[d] = run;
  }
  __syncthreads();
  {
    const uint32_t t = tid < RS_MAXDIG ? s_tot[tid] : 0u;
    const uint32_t ex = block_excl_scan<uint32_t>(t, nullptr);
    if (tid < RS_MAXDIG) s_start[tid] = ex;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RS_SUB; ++j) {
    const int64_t i = wbase + 32 * j + lane;
    if (i < n) {
      const uint32_t key = kk[j];
      const uint32_t d = (key >> shift) & dmask;
      const uint32_t pos = s_start[d] + s_cnt[w][d] + rnk[j];
      if (BP_DCHECK(pos < (uint32_t)RS_ITEMS, dbg, 201)) {
        s_k[pos] = key;
        s_v[pos] = vv[j];
      }
    }
  }
  __syncthreads();
  const int nvalid = (int)min((int64_t)RS_ITEMS, n - bbase);
  for (int p = tid; p < nvalid; p += RS_THREADS) {
    const uint32_t k = s_k[p];
    const uint32_t d = (k >> shift) & dmask;
    const int64_t g = s_off[d] + (p - (int64_t)s_start[d]);
    if (BP_DCHECK(g >= 0 && g < n, dbg, 202)) {
      kout[g] = k;
      vout[g] = s_v[p];
    }
  }
}

// start[t] = the first index whose key is >= t (t = 0 .. n_tiles; start[n_tiles] = n), by a
// binary search per key over the sorted keys: n_tiles + 1 threads, log2(n) reads each.
__global__ void k_tile_ranges(const uint32_t* __restrict__ keys, int64_t n, int64_t n_tiles,
                              int64_t* start) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t > n_tiles) return;
  int64_t lo = 0, hi = n;  // answer in [lo, hi]
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if ((int64_t)keys[mid] < t) lo = mid + 1; else hi = mid;
  }
  start[t] = lo;
}

// The scatter's 45 KB of shared memory per block: ask for the largest carveout, so that
// the four blocks its registers allow are resident together.
void rs_prefer_shared() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    cudaGetLastError();  // a preference only
    done = true;
  }
}

}  // namespace

// exclusive scan of n u32 counts into out[0..n-1]; out[n] receives the total.
int bp_scan_u32_to_i64(bp_ctx* ctx, const uint32_t* in, int64_t* out, int64_t n) {
  int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  if (nb == 0) nb = 1;
  int64_t* bsum;
  int r = bp_ws(ctx, WS_MISC, (size_t)(nb + 1) * sizeof(int64_t), (void**)&bsum);
  if (r) return r;
  k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, n, bsum);
  BP_LAUNCH_CHECK(ctx, "scan reduce");
  k_scan_bsums<<<1, SCAN_THREADS, 0, ctx->stream>>>(bsum, nb);
  BP_LAUNCH_CHECK(ctx, "scan block sums");
  k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, n, bsum, out);
  BP_LAUNCH_CHECK(ctx, "scan down");
  // total
  BP_CUDA(ctx, cudaMemcpyAsync(out + n, bsum + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                               ctx->stream));
  return BP_OK;
}

int bp_radix_sort_pairs(bp_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                        uint32_t* vals_tmp, int64_t n, int key_bits, uint32_t** keys_out,
                        uint32_t** vals_out) {
  *keys_out = keys;
  *vals_out = vals;
  if (n <= 1 || key_bits <= 0) return BP_OK;
  int64_t nblocks = (n + RS_ITEMS - 1) / RS_ITEMS;
  int npass = (key_bits + 7) / 8;
  int bits_per = (key_bits + npass - 1) / npass;  // balanced digit widths (<= 8)
  uint32_t* hist;
  int64_t* offs;
  int r = bp_ws(ctx, WS_HIST, (size_t)RS_MAXDIG * nblocks * sizeof(uint32_t) +
                                  ((size_t)RS_MAXDIG * nblocks + 1) * sizeof(int64_t) + 64,
                (void**)&hist);
  if (r) return r;
  offs = (int64_t*)(((uintptr_t)(hist + (size_t)RS_MAXDIG * nblocks) + 15) & ~(uintptr_t)15);
  uint32_t *ki = keys, *vi = vals, *ko = keys_tmp, *vo = vals_tmp;
  rs_prefer_shared();
  int shift = 0;
  for (int p = 0; p < npass; ++p) {
    int nb = (shift + bits_per <= key_bits) ? bits_per : key_bits - shift;
    int64_t hn = ((int64_t)1 << nb) * nblocks;
    k_rs_hist<<<(unsigned)nblocks, RS_THREADS, 0, ctx->stream>>>(ki, n, shift, nb, hist,
                                                                 nblocks);
    BP_LAUNCH_CHECK(ctx, "radix hist");
    r = bp_scan_u32_to_i64(ctx, hist, offs, hn);
    if (r) return r;
    k_rs_scatter<<<(unsigned)nblocks, RS_THREADS, 0, ctx->stream>>>(ki, vi, ko, vo, n, shift, nb,
                                                                    offs, nblocks,
                                                                    bp_dbg_word(ctx));
    BP_LAUNCH_CHECK(ctx, "radix scatter");
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    shift += nb;
  }
  *keys_out = ki;
  *vals_out = vi;
  return BP_OK;
}

int bp_tile_ranges(bp_ctx* ctx, const uint32_t* keys, int64_t n, int64_t n_tiles,
                   int64_t* tile_start) {
  int64_t threads = n_tiles + 1;
  k_tile_ranges<<<(unsigned)((threads + 255) / 256), 256, 0, ctx->stream>>>(keys, n, n_tiles,
                                                                            tile_start);
  BP_LAUNCH_CHECK(ctx, "tile ranges");
  return BP_OK;
}

// ---------------------------------------------------------------- caller-buffer variants
// Same kernels as above with every scratch buffer supplied by the caller (no bp_ws).
// bsum: >= (n / 8192 + 2) int64.
int bp_scan_u32_to_i64_buf(bp_ctx* ctx, const uint32_t* in, int64_t* out, int64_t n,
                           int64_t* bsum) {
  int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  if (nb == 0) nb = 1;
  k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, n, bsum);
  BP_LAUNCH_CHECK(ctx, "scan reduce");
  k_scan_bsums<<<1, SCAN_THREADS, 0, ctx->stream>>>(bsum, nb);
  BP_LAUNCH_CHECK(ctx, "scan block sums");
  k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, n, bsum, out);
  BP_LAUNCH_CHECK(ctx, "scan down");
  BP_CUDA(ctx, cudaMemcpyAsync(out + n, bsum + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                               ctx->stream));
  return BP_OK;
}

// hist: >= 256 * ceil(n / BP_RS_ITEMS) u32; offs: one more int64 than hist entries; bsum as
// above
int bp_radix_sort_pairs_buf(bp_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                            uint32_t* vals_tmp, int64_t n, int key_bits, uint32_t* hist,
                            int64_t* offs, int64_t* bsum, uint32_t** keys_out,
                            uint32_t** vals_out) {
  *keys_out = keys;
  *vals_out = vals;
  if (n <= 1 || key_bits <= 0) return BP_OK;
  int64_t nblocks = (n + RS_ITEMS - 1) / RS_ITEMS;
  int npass = (key_bits + 7) / 8;
  int bits_per = (key_bits + npass - 1) / npass;
  uint32_t *ki = keys, *vi = vals, *ko = keys_tmp, *vo = vals_tmp;
  rs_prefer_shared();
  int shift = 0, r;
  for (int p = 0; p < npass; ++p) {
    int nb = (shift + bits_per <= key_bits) ? bits_per : key_bits - shift;
    int64_t hn = ((int64_t)1 << nb) * nblocks;
    k_rs_hist<<<(unsigned)nblocks, RS_THREADS, 0, ctx->stream>>>(ki, n, shift, nb, hist,
                                                                 nblocks);
    BP_LAUNCH_CHECK(ctx, "radix hist");
    if ((r = bp_scan_u32_to_i64_buf(ctx, hist, offs, hn, bsum))) return r;
    k_rs_scatter<<<(unsigned)nblocks, RS_THREADS, 0, ctx->stream>>>(ki, vi, ko, vo, n, shift, nb,
                                                                    offs, nblocks,
                                                                    bp_dbg_word(ctx));
    BP_LAUNCH_CHECK(ctx, "radix scatter");
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    shift += nb;
  }
  *keys_out = ki;
  *vals_out = vi;
  return BP_OK;
}

// Loads the scan, radix-sort and tile-range kernels (CUDA loads modules lazily: a kernel's
// first launch would otherwise load its code into device memory).
int bp_sort_preload(bp_ctx* ctx) {
  cudaFuncAttributes a;
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_scan_reduce));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_scan_bsums));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_scan_down));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_rs_hist));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_rs_scatter));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_tile_ranges));
  return BP_OK;
}
