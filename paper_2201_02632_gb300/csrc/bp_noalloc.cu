// bp_noalloc.cu -- particle paste that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand their
// whole device memory to their own pool allocator at start-up (a simulation code that
// reserves HBM for its particle data, so a late cudaMalloc fails or fragments the
// pool), and latency-critical loops in which cudaMalloc/cudaFree would synchronise
// the device and stall the other streams.  bp_paste_particles_noalloc serves them: it
// runs the same pair list, radix sort and tiled deposit kernels as
// bp_paste_particles, with all of its scratch in the fixed file-scope device array
// below instead of the context's grow-on-demand buffers, and with one work unit per
// tile (no partial tiles).  CUDA loads a library's device code and arrays lazily, at their
// first use, and that load takes device memory; so bp_create does the set-up here
// (bp_noalloc_setup): it resolves the array's device address, which brings the array into
// being on the context's device, and loads every kernel this paste launches.  The array is
// then held until the process exits, and a later call allocates nothing.
#include <mutex>

#include "bp_internal.cuh"

namespace {

constexpr int64_t NA_MAX_PARTICLES = BP_NOALLOC_MAX_PARTICLES;
constexpr int64_t NA_MAX_PAIRS = BP_NOALLOC_MAX_PAIRS;
constexpr int64_t NA_MAX_TILES = BP_NOALLOC_MAX_TILES;
constexpr int64_t NA_RS_BLOCKS = (NA_MAX_PAIRS + BP_RS_ITEMS - 1) / BP_RS_ITEMS;
constexpr int64_t NA_HIST = 256 * NA_RS_BLOCKS;
constexpr int64_t NA_SCAN_MAX =
    (NA_MAX_PARTICLES > NA_HIST ? NA_MAX_PARTICLES : NA_HIST) > NA_MAX_TILES
        ? (NA_MAX_PARTICLES > NA_HIST ? NA_MAX_PARTICLES : NA_HIST)
        : NA_MAX_TILES;
constexpr int64_t NA_BSUM = NA_SCAN_MAX / 8192 + 2;

constexpr int64_t al(int64_t b) { return (b + 255) / 256 * 256; }
constexpr int64_t OFF_COUNTS = 0;
constexpr int64_t OFF_OFFS = OFF_COUNTS + al((NA_MAX_PARTICLES + 1) * 4);
constexpr int64_t OFF_K0 = OFF_OFFS + al((NA_MAX_PARTICLES + 1) * 8);
constexpr int64_t OFF_V0 = OFF_K0 + al(NA_MAX_PAIRS * 4);
constexpr int64_t OFF_K1 = OFF_V0 + al(NA_MAX_PAIRS * 4);
constexpr int64_t OFF_V1 = OFF_K1 + al(NA_MAX_PAIRS * 4);
constexpr int64_t OFF_HIST = OFF_V1 + al(NA_MAX_PAIRS * 4);
constexpr int64_t OFF_HOFFS = OFF_HIST + al(NA_HIST * 4);
constexpr int64_t OFF_BSUM = OFF_HOFFS + al((NA_HIST + 1) * 8);
constexpr int64_t OFF_TSTART = OFF_BSUM + al(NA_BSUM * 8);
constexpr int64_t OFF_UOFF = OFF_TSTART + al((NA_MAX_TILES + 1) * 8);
constexpr int64_t OFF_UCOUNT = OFF_UOFF + al((NA_MAX_TILES + 1) * 8);
constexpr int64_t OFF_UNITS = OFF_UCOUNT + al((NA_MAX_TILES + 1) * 4);
constexpr int64_t UNIT_BYTES_MAX = 32;  // checked against the real work-unit size
constexpr int64_t OFF_COUNTER = OFF_UNITS + al(NA_MAX_TILES * UNIT_BYTES_MAX);
constexpr int64_t NA_BYTES = OFF_COUNTER + 256;

// All scratch of every call on this device.  Calls share it: two calls whose work
// overlaps on the GPU (different streams, or different host threads) race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_setup_mutex;
void* g_scratch_ptr[64] = {nullptr};  // device address of the array, per device

// Device address of the array on the current device; looked up once per device.
int scratch_address(bp_ctx* ctx, unsigned char** out) {
  int dev = 0;
  BP_CUDA(ctx, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return bp_fail(ctx, BP_ERANGE, "paste (no allocation): device id");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return bp_fail(ctx, BP_ECUDA, "paste (no allocation): cudaGetSymbolAddress: %s",
                     cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_ptr[dev];
  return BP_OK;
}

}  // namespace

// Called by bp_create with the context's device current: the array's address and the kernels
// of the paste, so that bp_paste_particles_noalloc itself loads nothing.  A device id the
// table cannot hold is left to the paste call, which reports it.
int bp_noalloc_setup(bp_ctx* ctx) {
  int dev = 0;
  BP_CUDA(ctx, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return BP_OK;
  unsigned char* base = nullptr;
  int r;
  if ((r = scratch_address(ctx, &base))) return r;
  if ((r = bp_pp_preload(ctx))) return r;
  if ((r = bp_sort_preload(ctx))) return r;
  return bp_deposit_tc_preload(ctx);
}

extern "C" int bp_paste_particles_noalloc(bp_ctx* ctx, int64_t n, const float* assigned,
                                          const bp_map_geom* geom, int select, float* ymap,
                                          float* bmap, float* ylo, float* blo) {
  if (!ctx) return BP_EINVAL;
  if (!geom || geom->nx <= 0 || geom->ny <= 0 || geom->n_maps != 1 || !(geom->dtheta > 0))
    return bp_fail(ctx, BP_EINVAL, "paste (no allocation): bad geometry (n_maps must be 1)");
  if (geom->nx > 65536 || geom->ny > 65536)
    return bp_fail(ctx, BP_ERANGE, "paste (no allocation): map side above 65536 pixels");
  if (n < 0) return bp_fail(ctx, BP_EINVAL, "paste (no allocation): n < 0");
  if (n > NA_MAX_PARTICLES)
    return bp_fail(ctx, BP_ERANGE, "paste (no allocation): %lld particles exceed the limit %lld",
                   (long long)n, (long long)NA_MAX_PARTICLES);
  if (select < 0 || select > 2) return bp_fail(ctx, BP_EINVAL, "paste (no allocation): select");
  if (n == 0) return BP_OK;
  if (!assigned || !ymap || !bmap || !ylo || !blo)
    return bp_fail(ctx, BP_EINVAL, "paste (no allocation): null pointer");
  if (((uintptr_t)assigned & 15) != 0)
    return bp_fail(ctx, BP_EINVAL, "paste (no allocation): records must be 16-byte aligned");
  if ((int64_t)bp_pp_unit_bytes() > UNIT_BYTES_MAX)
    return bp_fail(ctx, BP_ECUDA, "paste (no allocation): work-unit record too large");
  unsigned char* base = nullptr;
  int r = scratch_address(ctx, &base);
  if (r) return r;
  BpPasteBuffers B;
  B.counts = (uint32_t*)(base + OFF_COUNTS);
  B.offs = (int64_t*)(base + OFF_OFFS);
  B.keys0 = (uint32_t*)(base + OFF_K0);
  B.vals0 = (uint32_t*)(base + OFF_V0);
  B.keys1 = (uint32_t*)(base + OFF_K1);
  B.vals1 = (uint32_t*)(base + OFF_V1);
  B.hist = (uint32_t*)(base + OFF_HIST);
  B.hoffs = (int64_t*)(base + OFF_HOFFS);
  B.bsum = (int64_t*)(base + OFF_BSUM);
  B.tstart = (int64_t*)(base + OFF_TSTART);
  B.uoff = (int64_t*)(base + OFF_UOFF);
  B.ucount = (uint32_t*)(base + OFF_UCOUNT);
  B.units = (void*)(base + OFF_UNITS);
  B.counter = (int64_t*)(base + OFF_COUNTER);  // cleared inside before the deposit
  B.max_pairs = NA_MAX_PAIRS;
  B.max_tiles = NA_MAX_TILES;
  return bp_pp_paste_buffers(ctx, n, assigned, geom, select, ymap, bmap, ylo, blo, &B);
}
