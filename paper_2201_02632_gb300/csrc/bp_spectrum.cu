// bp_spectrum.cu -- angular power spectrum of a flat-sky map (Section 5.3: the FFT of the map,
// binned in logarithmic multipole bins).
//
//   a(l) = dtheta^2 sum_pixels f(theta) e^{-i l.theta},  C(l) = |a(l)|^2 / (nx ny dtheta^2),
//   l = 2 pi (kx / (nx dtheta), ky / (ny dtheta)) for the integer frequencies kx, ky,
// averaged over the modes whose |l| falls in each bin [edges[b], edges[b+1]).
//
//  k_fft_rows     one CTA per map row: FP32 map (+ lo plane) -> FP64 complex, radix-2
//                 decimation-in-time FFT in shared memory (bit-reversed load, log2 n stages
//                 with host FP64 twiddles), written row-major
//  k_transpose    32 x 32 shared-memory tiles: the columns become rows
//  k_fft_bin      one CTA per former column (frequency kx): the same FFT along y, then every
//                 mode's power and bin (FP64, explicitly rounded |l|^2 against the squared
//                 edges), and per-bin sums of the row in a fixed lane / shuffle order
//  k_bin_reduce   per bin: the row partials summed in a fixed tree, divided by the mode count
//
// Everything is FP64 (the FFT costs ~5 n log2 n flops per map, small next to the pastes), so
// the bins agree with an FP64 reference to rounding and each mode's bin is decided exactly
// as the reference decides it.
#include <cmath>
#include <vector>

#include "bp_internal.cuh"

namespace {

constexpr int FT_THREADS = 512;
constexpr int MAX_BINS = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place FFT of s[0..n) (already in bit-reversed order), twiddles w[j] = e^{-2 pi i j / n}.
__device__ __forceinline__ void fft_smem(double2* s, int n, const double2* __restrict__ w) {
  for (int half = 1, lg = 0; half < n; half <<= 1, ++lg) {
    const int stride = n / (2 * half);
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int j = b & (half - 1);
      const int i0 = ((b >> lg) << (lg + 1)) + j, i1 = i0 + half;
      const double2 u = s[i0], v = cmul(s[i1], __ldg(w + j * stride));
      s[i0] = make_double2(u.x + v.x, u.y + v.y);
      s[i1] = make_double2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(FT_THREADS)
    k_fft_rows(const float* __restrict__ map, const float* __restrict__ lo, int nx, int lgx,
               const double2* __restrict__ wx, double2* out) {
  extern __shared__ double2 s_c[];
  const int64_t row = blockIdx.x;
  const float* m = map + row * nx;
  const float* l = lo ? lo + row * nx : nullptr;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double v = (double)m[i] + (l ? (double)l[i] : 0.0);
    s_c[__brev((unsigned)i) >> (32 - lgx)] = make_double2(v, 0.0);
  }
  __syncthreads();
  fft_smem(s_c, nx, wx);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) out[row * nx + i] = s_c[i];
}

// in [rows][cols] -> out [cols][rows]
__global__ void k_transpose(const double2* __restrict__ in, int rows, int cols, double2* out) {
  __shared__ double2 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[k][threadIdx.x] = in[(int64_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(int64_t)c * rows + r] = t[threadIdx.x][k];
  }
}

// Row kx of the transposed spectrum: FFT along y, then per-bin sums of the row's power.
__global__ void __launch_bounds__(FT_THREADS)
    k_fft_bin(const double2* __restrict__ in, int nx, int ny, int lgy,
              const double2* __restrict__ wy, double inv_lx, double inv_ly, double c2,
              double norm, const double* __restrict__ edges2, int nb, double* psum,
              int* pcnt) {
  extern __shared__ double2 s_c[];
  __shared__ double s_e2[MAX_BINS + 1];
  short* s_bin = reinterpret_cast<short*>(s_c + ny);
  const int kx = blockIdx.x;
  for (int i = threadIdx.x; i <= nb; i += blockDim.x) s_e2[i] = edges2[i];
  for (int i = threadIdx.x; i < ny; i += blockDim.x)
    s_c[__brev((unsigned)i) >> (32 - lgy)] = in[(int64_t)kx * ny + i];
  __syncthreads();
  fft_smem(s_c, ny, wy);
  // |l|^2 = c2 ((kx / Lx)^2 + (ky / Ly)^2), every operation rounded as written
  const int fx = kx < nx / 2 ? kx : kx - nx;
  const double ux = __dmul_rn((double)fx, inv_lx);
  const double ux2 = __dmul_rn(ux, ux);
  for (int i = threadIdx.x; i < ny; i += blockDim.x) {
    const int fy = i < ny / 2 ? i : i - ny;
    const double uy = __dmul_rn((double)fy, inv_ly);
    const double l2 = __dmul_rn(c2, __dadd_rn(ux2, __dmul_rn(uy, uy)));
    int b = -1;
    if (l2 >= s_e2[0] && l2 < s_e2[nb]) {
      int lo = 0, hi = nb - 1;  // last edge <= l2
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_e2[mid] <= l2) lo = mid; else hi = mid - 1;
      }
      b = lo;
    }
    const double2 v = s_c[i];
    s_c[i].x = __dmul_rn(norm, __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)));
    s_bin[i] = (short)b;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = wid; b < nb; b += nw) {
    double s = 0.0;
    int c = 0;
    for (int i = lane; i < ny; i += 32)
      if (s_bin[i] == b) {
        s += s_c[i].x;
        ++c;
      }
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      psum[(int64_t)kx * nb + b] = s;
      pcnt[(int64_t)kx * nb + b] = c;
    }
  }
}

// One block per bin: rows summed lane-strided, then a fixed shared-memory tree (the same
// order on every run).
constexpr int BR_THREADS = 256;
__global__ void __launch_bounds__(BR_THREADS)
    k_bin_reduce(const double* __restrict__ psum, const int* __restrict__ pcnt, int nrows, int nb,
                 double* cl, int64_t* nmodes) {
  __shared__ double s_s[BR_THREADS];
  __shared__ long long s_c[BR_THREADS];
  const int b = blockIdx.x, t = threadIdx.x;
  double s = 0.0;
  long long c = 0;
  for (int r = t; r < nrows; r += BR_THREADS) {
    s += psum[(int64_t)r * nb + b];
    c += pcnt[(int64_t)r * nb + b];
  }
  s_s[t] = s;
  s_c[t] = c;
  __syncthreads();
  for (int o = BR_THREADS / 2; o > 0; o >>= 1) {
    if (t < o) {
      s_s[t] += s_s[t + o];
      s_c[t] += s_c[t + o];
    }
    __syncthreads();
  }
  if (t == 0) {
    cl[b] = s_c[0] > 0 ? s_s[0] / (double)s_c[0] : 0.0;
    if (nmodes) nmodes[b] = s_c[0];
  }
}

int log2_exact(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return (1 << l) == n ? l : -1;
}

}  // namespace

extern "C" int bp_power_spectrum(bp_ctx* ctx, const float* map, const float* lo, int nx, int ny,
                                 double dtheta, int nb, const double* edges, double* cl,
                                 int64_t* nmodes) {
  if (!ctx) return BP_EINVAL;
  const int lgx = log2_exact(nx), lgy = log2_exact(ny);
  if (lgx < 1 || lgy < 1 || nx > 8192 || ny > 8192)
    return bp_fail(ctx, BP_EINVAL, "bp_power_spectrum: nx, ny must be powers of two in [2, 8192]");
  if (!(dtheta > 0)) return bp_fail(ctx, BP_EINVAL, "bp_power_spectrum: dtheta <= 0");
  if (nb < 1 || nb > MAX_BINS) return bp_fail(ctx, BP_EINVAL, "bp_power_spectrum: nb outside [1, 256]");
  if (!map || !edges || !cl) return bp_fail(ctx, BP_EINVAL, "bp_power_spectrum: null pointer");
  for (int b = 0; b < nb; ++b)
    if (!(edges[b] >= 0.0) || !(edges[b + 1] > edges[b]))
      return bp_fail(ctx, BP_EINVAL, "bp_power_spectrum: edges must increase from >= 0");
  int r;
  const size_t ncell = (size_t)nx * ny;
  double2 *A, *B;
  if ((r = bp_ws(ctx, WS_PART, ncell * sizeof(double2), (void**)&A))) return r;
  if ((r = bp_ws(ctx, WS_TABLE, ncell * sizeof(double2), (void**)&B))) return r;
  // twiddles (both axes), squared edges, row partials
  const size_t nw = (size_t)(nx / 2 + ny / 2);
  const size_t small = nw * sizeof(double2) + (size_t)(nb + 1) * 8;
  char* S;
  if ((r = bp_ws(ctx, WS_MISC2, small, (void**)&S))) return r;
  double* psum;
  if ((r = bp_ws(ctx, WS_MISC3, (size_t)nx * nb * (8 + 4), (void**)&psum))) return r;
  int* pcnt = reinterpret_cast<int*>(psum + (size_t)nx * nb);
  std::vector<char> host(small);
  double2* hw = reinterpret_cast<double2*>(host.data());
  for (int j = 0; j < nx / 2; ++j)
    hw[j] = make_double2(cos(-2.0 * bpc::PI * j / nx), sin(-2.0 * bpc::PI * j / nx));
  for (int j = 0; j < ny / 2; ++j)
    hw[nx / 2 + j] = make_double2(cos(-2.0 * bpc::PI * j / ny), sin(-2.0 * bpc::PI * j / ny));
  double* he2 = reinterpret_cast<double*>(hw + nw);
  for (int b = 0; b <= nb; ++b) he2[b] = edges[b] * edges[b];
  BP_CUDA(ctx, cudaMemcpyAsync(S, host.data(), small, cudaMemcpyHostToDevice, ctx->stream));
  // the host copy must stay alive until the copy has run
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const double2* wx = reinterpret_cast<const double2*>(S);
  const double2* wy = wx + nx / 2;
  const double* e2 = reinterpret_cast<const double*>(wx + nw);
  const int tx = std::min(FT_THREADS, std::max(32, nx / 2));
  const int ty = std::min(FT_THREADS, std::max(32, ny / 2));
  const size_t smx = (size_t)nx * sizeof(double2);
  const size_t smy = (size_t)ny * (sizeof(double2) + sizeof(short));
  BP_CUDA(ctx, cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx));
  BP_CUDA(ctx, cudaFuncSetAttribute(k_fft_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy));
  k_fft_rows<<<ny, tx, smx, ctx->stream>>>(map, lo, nx, lgx, wx, A);
  BP_LAUNCH_CHECK(ctx, "fft rows");
  k_transpose<<<dim3((nx + 31) / 32, (ny + 31) / 32), dim3(32, 8), 0, ctx->stream>>>(A, ny, nx, B);
  BP_LAUNCH_CHECK(ctx, "fft transpose");
  const double inv_lx = 1.0 / (nx * dtheta), inv_ly = 1.0 / (ny * dtheta);
  const double c2 = 4.0 * bpc::PI * bpc::PI;
  const double norm = dtheta * dtheta / (double)ncell;
  k_fft_bin<<<nx, ty, smy, ctx->stream>>>(B, nx, ny, lgy, wy, inv_lx, inv_ly, c2, norm, e2, nb,
                                          psum, pcnt);
  BP_LAUNCH_CHECK(ctx, "fft bins");
  k_bin_reduce<<<nb, BR_THREADS, 0, ctx->stream>>>(psum, pcnt, nx, nb, cl, nmodes);
  BP_LAUNCH_CHECK(ctx, "bin reduce");
  return BP_OK;
}
