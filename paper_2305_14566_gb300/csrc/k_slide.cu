// Slide preparation (Sec. 2.1 of the paper): padding with the 2x2-mean colour,
// the 40x -> 20x -> 10x -> 5x pyramid (Sec. 2.2), the 32x tissue thumbnail,
// median blur, Otsu threshold, tissue mask and the foreground tile lists.
// Everything here is integer arithmetic and bit-exact by construction.
#include "omni_internal.cuh"

namespace omni {
namespace {

// ------------------------------------------------------------------ synthetic slides
// Input generator only (not part of the method): SplitMix64 (Steele, Lea &
// Flood 2014; mixer constants as published by Vigna) over pixel counters and
// integer rotated-ellipse tissue.

struct EllParams {
  int n;
  long long e[kMaxEll][6];   // cy, cx, a, b, cos_q14, sin_q14
};

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long idx) {
  unsigned long long z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Sharp-edged structure discs inside needle cores: one 512 x 512 cell per
// SplitMix64 draw (seed ^ kStructSalt, index cell_row << 20 | cell_col);
// returns the disc type 0..2 covering (gy, gx), or -1.
constexpr unsigned long long kStructSalt = 0x5A17C0DE5EEDull;
__device__ __forceinline__ int structure_at(unsigned long long seed, long long gy, long long gx) {
  const long long cy = gy >> 9, cx = gx >> 9;
  const unsigned long long h = splitmix64(seed ^ kStructSalt, (unsigned long long)((cy << 20) | cx));
  if ((long long)(h & 0xFF) >= 160) return -1;
  const long long r = 64 + (long long)((h >> 16) & 0x7F), m = 254 - r;
  const long long ccy = (cy << 9) + 256 + ((long long)((h >> 24) & 0xFF) * 2 * m) / 255 - m;
  const long long ccx = (cx << 9) + 256 + ((long long)((h >> 32) & 0xFF) * 2 * m) / 255 - m;
  const long long dy = gy - ccy, dx = gx - ccx;
  return dy * dy + dx * dx < r * r ? (int)(((h >> 8) & 0xFF) % 3) : -1;
}

__global__ void k_synth(EllParams ep, unsigned long long seed, int structures, int slide_w, int y0, int x0,
                        int h, int w, uint8_t* out, long long stride) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= w || y >= h) return;
  long long gy = y0 + y, gx = x0 + x;
  long long depth = -1;
  for (int k = 0; k < ep.n; ++k) {
    const long long* e = ep.e[k];
    long long dy = gy - e[0], dx = gx - e[1];
    long long u = dx * e[4] + dy * e[5];
    long long v = -dx * e[5] + dy * e[4];
    u = u < 0 ? -u : u;
    v = v < 0 ? -v : v;
    long long uq = (u << 2) / e[2];
    long long vq = (v << 2) / e[3];
    uq = uq < (1ll << 20) ? uq : (1ll << 20);
    vq = vq < (1ll << 20) ? vq : (1ll << 20);
    long long r = uq * uq + vq * vq;
    if (r < (1ll << 32)) {
      long long t8 = ((1ll << 32) - r) >> 24;
      if (t8 > depth) depth = t8;
    }
  }
  const int pink[3] = {232, 150, 200}, purple[3] = {150, 90, 170};
  const int scol[3][3] = {{120, 50, 140}, {245, 205, 230}, {195, 65, 95}};
  const int st = structures && depth >= 0 ? structure_at(seed, gy, gx) : -1;
  unsigned long long base = ((unsigned long long)gy * (unsigned long long)slide_w +
                             (unsigned long long)gx) * 3ull;
  uint8_t* o = out + (long long)y * stride + (long long)x * 3;
  for (int c = 0; c < 3; ++c) {
    unsigned long long hsh = splitmix64(seed, base + c);
    long long s = (long long)(hsh & 0xFFFF) + (long long)((hsh >> 16) & 0xFFFF) +
                  (long long)((hsh >> 32) & 0xFFFF) + (long long)((hsh >> 48) & 0xFFFF);
    long long noise = ((s * 10 - 1310700 + 32768 + (32ll << 16)) >> 16) - 32;
    long long t = depth > 0 ? depth : 0;
    long long col = depth >= 0 ? ((pink[c] * (256 - t) + purple[c] * t + 128) >> 8) : 235;
    if (st >= 0) col = scol[st][c];
    long long val = col + noise;
    val = val < 0 ? 0 : (val > 255 ? 255 : val);
    o[c] = (uint8_t)val;
  }
}

// ------------------------------------------------------------------ padding
__global__ void k_pad(const uint8_t* __restrict__ rgb, long long stride, SlideGeom g,
                      uint8_t* __restrict__ canvas) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= g.Wp) return;
  int sy = y - g.lead, sx = x - g.lead;
  uint8_t* o = canvas + ((long long)y * g.Wp + x) * 3;
  if (sy >= 0 && sy < g.H && sx >= 0 && sx < g.W) {
    const uint8_t* p = rgb + (long long)sy * stride + (long long)sx * 3;
    o[0] = p[0]; o[1] = p[1]; o[2] = p[2];
  } else {
    // Sec. 2.1: pad colour = rounded mean of the 2x2 top-left pixels
    int h2 = g.H > 1 ? 2 : 1, w2 = g.W > 1 ? 2 : 1;
    for (int c = 0; c < 3; ++c) {
      int s = 0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          s += rgb[(long long)(a < h2 ? a : 0) * stride + (b < w2 ? b : 0) * 3 + c];
      o[c] = (uint8_t)((s + 2) >> 2);
    }
  }
}

// ------------------------------------------------------------------ pyramid
// One thread per 8x8 block of 40x pixels: iterated 2x2 means (round half up)
// give its 4x4 20x, 2x2 10x and 1x1 5x pixels; the raw 8x8 sums feed the
// thumbnail.
__global__ void k_pyramid(const uint8_t* __restrict__ c40, long long s40, int Hp, int Wp,
                          uint8_t* __restrict__ c20, uint8_t* __restrict__ c10,
                          uint8_t* __restrict__ c5, uint16_t* __restrict__ blk8) {
  int bx = blockIdx.x * blockDim.x + threadIdx.x;
  int by = blockIdx.y;
  int nbx = Wp >> 3;
  if (bx >= nbx) return;
  int sum[3] = {0, 0, 0};
  int h20[4][4][3];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int v[2][8][3];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const uint2* row = reinterpret_cast<const uint2*>(
          c40 + (long long)(by * 8 + 2 * r + rr) * s40 + (long long)bx * 24);
      uint2 q0 = __ldg(row), q1 = __ldg(row + 1), q2 = __ldg(row + 2);
      uint32_t w[6] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y};
#pragma unroll
      for (int i = 0; i < 24; ++i) v[rr][i / 3][i % 3] = (w[i >> 2] >> ((i & 3) * 8)) & 0xFF;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        int s4 = v[0][2 * q][c] + v[0][2 * q + 1][c] + v[1][2 * q][c] + v[1][2 * q + 1][c];
        sum[c] += s4;
        h20[r][q][c] = (s4 + 2) >> 2;
      }
  }
  int nb = (by * nbx + bx) * 3;
  blk8[nb + 0] = (uint16_t)sum[0];
  blk8[nb + 1] = (uint16_t)sum[1];
  blk8[nb + 2] = (uint16_t)sum[2];
  if (c20) {
    long long s20 = (long long)(Wp / 2) * 3;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          c20[(long long)(by * 4 + r) * s20 + (bx * 4 + q) * 3 + c] = (uint8_t)h20[r][q][c];
  }
  int h10[2][2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        h10[r][q][c] = (h20[2 * r][2 * q][c] + h20[2 * r][2 * q + 1][c] +
                        h20[2 * r + 1][2 * q][c] + h20[2 * r + 1][2 * q + 1][c] + 2) >> 2;
  if (c10) {
    long long s10 = (long long)(Wp / 4) * 3;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          c10[(long long)(by * 2 + r) * s10 + (bx * 2 + q) * 3 + c] = (uint8_t)h10[r][q][c];
  }
  if (c5) {
    long long s5 = (long long)(Wp / 8) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      c5[(long long)by * s5 + bx * 3 + c] =
          (uint8_t)((h10[0][0][c] + h10[0][1][c] + h10[1][0][c] + h10[1][1][c] + 2) >> 2);
  }
}

// ------------------------------------------------------------------ tissue mask
// thumbnail pixel = (sum of its 32x32 40x pixels + 512) >> 10; grey =
// (77 R + 150 G + 29 B + 128) >> 8
__global__ void k_thumb_grey(const uint16_t* __restrict__ blk8, int nbx, int th, int tw,
                             uint8_t* __restrict__ grey) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= tw) return;
  int s[3] = {0, 0, 0};
  for (int r = 0; r < 4; ++r)
    for (int q = 0; q < 4; ++q) {
      const uint16_t* b = blk8 + ((long long)(y * 4 + r) * nbx + (x * 4 + q)) * 3;
      s[0] += b[0]; s[1] += b[1]; s[2] += b[2];
    }
  int R = (s[0] + 512) >> 10, G = (s[1] + 512) >> 10, B = (s[2] + 512) >> 10;
  grey[y * tw + x] = (uint8_t)((77 * R + 150 * G + 29 * B + 128) >> 8);
}

// k x k median with replicated borders.  One thread per column keeps a
// 256-bin histogram of its window and slides it down a strip of rows; the
// median is the smallest level whose cumulative count reaches (k*k + 1) / 2.
constexpr int kMedStrip = 32;
__global__ void __launch_bounds__(32) k_median(const uint8_t* __restrict__ grey, int th, int tw,
                                               int k, uint8_t* __restrict__ out) {
  __shared__ uint32_t hist[256][32];
  int t = threadIdx.x;
  int x = blockIdx.x * 32 + t;
  int y0 = blockIdx.y * kMedStrip;
  int y1 = min(th, y0 + kMedStrip);
  for (int v = 0; v < 256; ++v) hist[v][t] = 0;
  if (x >= tw) return;
  int r = k >> 1;
  int need = (k * k + 1) >> 1;
  for (int dy = -r; dy <= r; ++dy) {
    int yy = min(max(y0 + dy, 0), th - 1);
    for (int dx = -r; dx <= r; ++dx) {
      int xx = min(max(x + dx, 0), tw - 1);
      hist[grey[yy * tw + xx]][t] += 1;
    }
  }
  for (int y = y0; y < y1; ++y) {
    if (y > y0) {
      int yo = min(max(y - 1 - r, 0), th - 1), yi = min(max(y + r, 0), th - 1);
      for (int dx = -r; dx <= r; ++dx) {
        int xx = min(max(x + dx, 0), tw - 1);
        hist[grey[yo * tw + xx]][t] -= 1;
        hist[grey[yi * tw + xx]][t] += 1;
      }
    }
    int cnt = 0, med = 255;
    for (int v = 0; v < 256; ++v) {
      cnt += hist[v][t];
      if (cnt >= need) { med = v; break; }
    }
    out[y * tw + x] = (uint8_t)med;
  }
}

__global__ void k_hist(const uint8_t* __restrict__ img, long long n, int32_t* __restrict__ hist) {
  __shared__ int32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    atomicAdd(&h[img[i]], 1);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Otsu on 256 bins, exact.  Score(t) = (N S(t) - W(t) S_T)^2 / (W(t) (N - W(t)))
// is compared as quotient + remainder so every product fits in 128 bits.
// Ties go to the smallest t; splits with W = 0 or W = N are skipped.
struct OtsuKey {
  unsigned __int128 q;
  unsigned long long r, d;
  int t;
};
__device__ __forceinline__ bool otsu_better(const OtsuKey& a, const OtsuKey& b) {
  // is a strictly better than b (or equal and with a smaller t)?
  if (a.t < 0) return false;
  if (b.t < 0) return true;
  if (a.q != b.q) return a.q > b.q;
  unsigned __int128 l = (unsigned __int128)a.r * b.d, rr = (unsigned __int128)b.r * a.d;
  if (l != rr) return l > rr;
  return a.t < b.t;
}

__global__ void __launch_bounds__(256) k_otsu(const int32_t* __restrict__ hist,
                                              int32_t* __restrict__ out) {
  __shared__ unsigned long long W[256], S[256];
  __shared__ OtsuKey key[256];
  int t = threadIdx.x;
  W[t] = (unsigned long long)hist[t];
  S[t] = (unsigned long long)hist[t] * (unsigned long long)t;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    unsigned long long w = t >= off ? W[t - off] : 0, s = t >= off ? S[t - off] : 0;
    __syncthreads();
    W[t] += w;
    S[t] += s;
    __syncthreads();
  }
  unsigned long long N = W[255], ST = S[255], w = W[t], s = S[t];
  OtsuKey k;
  k.t = -1; k.q = 0; k.r = 0; k.d = 1;
  if (w != 0 && w != N) {
    unsigned long long a = N * s, b = w * ST;
    unsigned long long diff = a > b ? a - b : b - a;
    unsigned __int128 num = (unsigned __int128)diff * diff;
    unsigned long long den = w * (N - w);
    k.q = num / den;
    k.r = (unsigned long long)(num % den);
    k.d = den;
    k.t = t;
  }
  key[t] = k;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (t < off && otsu_better(key[t + off], key[t])) key[t] = key[t + off];
    __syncthreads();
  }
  if (t == 0) out[0] = key[0].t;
}

__global__ void k_mask(const uint8_t* __restrict__ blurred, long long n,
                       const int32_t* __restrict__ otsu, uint8_t* __restrict__ mask) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  mask[i] = (int)blurred[i] <= otsu[0] ? 1 : 0;
}

// ------------------------------------------------------------------ tile lists
// A tile of scale s at grid (i, j) covers thumbnail rows i*S_s*f/32 ..
// (i*S_s+P)*f/32 - 1 (and the same for columns); it is foreground when any
// tissue pixel lies there.
__global__ void k_tile_flags(const uint8_t* __restrict__ mask, SlideGeom g, int filter,
                             uint8_t* __restrict__ flags) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int total = g.grid_off[g.n_scales];
  if (idx >= total) return;
  int s = 0;
  while (idx >= g.grid_off[s + 1]) ++s;
  int cell = idx - g.grid_off[s];
  int i = cell / g.gw[s], j = cell % g.gw[s];
  uint8_t fg = 1;
  if (filter) {
    int f = g.factors[s];
    const int S = g.S[s];
    int r0 = i * S * f / kThumb, r1 = (i * S + g.P) * f / kThumb;
    int c0 = j * S * f / kThumb, c1 = (j * S + g.P) * f / kThumb;
    fg = 0;
    for (int r = r0; r < r1 && !fg; ++r)
      for (int c = c0; c < c1; ++c)
        if (mask[r * g.tw + c]) { fg = 1; break; }
  }
  flags[idx] = fg;
}

// Stable compaction of every scale's flag grid (one block, chunks of 1024).
__global__ void __launch_bounds__(1024) k_tile_compact(const uint8_t* __restrict__ flags,
                                                       SlideGeom g, int32_t* __restrict__ tiles,
                                                       int32_t* __restrict__ counts,
                                                       int32_t* __restrict__ slot_map) {
  __shared__ int scan[1024];
  __shared__ int carry_s;
  int t = threadIdx.x;
  int total_count = 0;
  for (int s = 0; s < g.n_scales; ++s) {
    int n = g.gh[s] * g.gw[s];
    int base = g.grid_off[s];
    if (t == 0) carry_s = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += 1024) {
      int cell = c0 + t;
      int f = cell < n ? flags[base + cell] : 0;
      scan[t] = f;
      __syncthreads();
      for (int off = 1; off < 1024; off <<= 1) {
        int v = t >= off ? scan[t - off] : 0;
        __syncthreads();
        scan[t] += v;
        __syncthreads();
      }
      int carry = carry_s;
      if (cell < n) {
        int pos = carry + scan[t] - f;         // index within this scale
        slot_map[base + cell] = f ? pos : -1;
        if (f) {
          int o = total_count + pos;
          tiles[o * 3 + 0] = s;
          tiles[o * 3 + 1] = (cell / g.gw[s]) * g.S[s];
          tiles[o * 3 + 2] = (cell % g.gw[s]) * g.S[s];
        }
      }
      __syncthreads();
      if (t == 1023) carry_s = carry + scan[1023];
      __syncthreads();
    }
    if (t == 0) counts[1 + s] = carry_s;
    total_count += carry_s;
    __syncthreads();
  }
  if (t == 0) counts[0] = total_count;
}

}  // namespace

cudaError_t launch_synth(const int64_t* ell_host, int n_ell, uint64_t seed, int structures, int slide_w,
                         int y0, int x0, int h, int w, uint8_t* out, int64_t stride, cudaStream_t st) {
  if (n_ell < 0 || n_ell > kMaxEll) return cudaErrorInvalidValue;
  EllParams ep;
  ep.n = n_ell;
  for (int k = 0; k < n_ell; ++k)
    for (int q = 0; q < 6; ++q) ep.e[k][q] = ell_host[k * 6 + q];
  if (h <= 0 || w <= 0) return cudaSuccess;
  dim3 grid((w + 255) / 256, h);
  k_synth<<<grid, 256, 0, st>>>(ep, seed, structures, slide_w, y0, x0, h, w, out, stride);
  return cudaGetLastError();
}

cudaError_t launch_pad(const uint8_t* rgb, int64_t stride, const SlideGeom& g, uint8_t* canvas,
                       cudaStream_t st) {
  dim3 grid((g.Wp + 255) / 256, g.Hp);
  k_pad<<<grid, 256, 0, st>>>(rgb, stride, g, canvas);
  return cudaGetLastError();
}

cudaError_t launch_pyramid(const uint8_t* c40, int64_t stride40, int Hp, int Wp, uint8_t* c20,
                           uint8_t* c10, uint8_t* c5, uint16_t* blk8, cudaStream_t st) {
  int nbx = Wp / 8, nby = Hp / 8;
  dim3 grid((nbx + 63) / 64, nby);
  k_pyramid<<<grid, 64, 0, st>>>(c40, stride40, Hp, Wp, c20, c10, c5, blk8);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ area filter
// Sec. 2.1 contour step: tissue regions are the 8-connected components of the
// thumbnail mask; regions of fewer than min_area pixels are cleared.  The
// components come from a concurrent union-find over the mask: a label points
// to a smaller pixel index until the root (the region's smallest index);
// every tissue pixel unites with its tissue neighbours to the west,
// north-west, north and north-east (the other four directions are those
// pixels' own unions).  A union relinks the larger root below the smaller
// with atomicMin and retries with whatever the larger root had become, so
// labels only decrease and every loop ends; each loop also stops after n
// steps with an error bit (it cannot need more).
__device__ __forceinline__ int ccl_find(const volatile int32_t* L, int x, int n, bool& ok) {
  for (int k = 0; k < n; ++k) {
    const int y = L[x];
    if (y == x) return x;
    x = y;
  }
  ok = false;
  return x;
}

__device__ __forceinline__ bool ccl_unite(int32_t* L, int a, int b, int n) {
  bool ok = true;
  for (int k = 0; k < n && ok; ++k) {
    a = ccl_find(L, a, n, ok);
    b = ccl_find(L, b, n, ok);
    if (!ok || a == b) return ok;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(&L[b], a);
    if (old == b) return true;      // b was a root and now hangs below a
    b = old;                        // b had been relinked meanwhile: join a with its new parent
  }
  return false;
}

__global__ void k_ccl_init(const uint8_t* __restrict__ mask, int n, int32_t* __restrict__ L,
                           int32_t* __restrict__ area) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  L[i] = mask[i] ? i : -1;
  area[i] = 0;
}

__global__ void k_ccl_union(const uint8_t* __restrict__ mask, int th, int tw, int32_t* L, unsigned* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = th * tw;
  if (i >= n || !mask[i]) return;
  const int y = i / tw, x = i - y * tw;
  bool ok = true;
  if (x > 0 && mask[i - 1]) ok &= ccl_unite(L, i, i - 1, n);
  if (y > 0) {
    const int up = i - tw;
    if (x > 0 && mask[up - 1]) ok &= ccl_unite(L, i, up - 1, n);
    if (mask[up]) ok &= ccl_unite(L, i, up, n);
    if (x + 1 < tw && mask[up + 1]) ok &= ccl_unite(L, i, up + 1, n);
  }
  if (!ok) atomicOr(err, kErrTimeout);
}

// every tissue pixel's label becomes its region's root; the root counts it
__global__ void k_ccl_count(const uint8_t* __restrict__ mask, int n, int32_t* L, int32_t* area,
                            unsigned* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !mask[i]) return;
  bool ok = true;
  const int r = ccl_find(L, i, n, ok);
  if (!ok) atomicOr(err, kErrTimeout);
  L[i] = r;
  atomicAdd(&area[r], 1);
}

__global__ void k_ccl_apply(uint8_t* __restrict__ mask, int n, const int32_t* __restrict__ L,
                            const int32_t* __restrict__ area, int min_area) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !mask[i]) return;
  if (area[L[i]] < min_area) mask[i] = 0;
}

cudaError_t launch_area_filter(uint8_t* mask, int th, int tw, int min_area, int32_t* region, int32_t* area,
                               unsigned* err, cudaStream_t st) {
  if (min_area <= 0) return cudaSuccess;
  if (th <= 0 || tw <= 0 || (long long)th * tw > (1LL << 30)) return cudaErrorInvalidValue;
  const int n = th * tw;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_ccl_init<<<blocks, 256, 0, st>>>(mask, n, region, area);
  k_ccl_union<<<blocks, 256, 0, st>>>(mask, th, tw, region, err);
  k_ccl_count<<<blocks, 256, 0, st>>>(mask, n, region, area, err);
  k_ccl_apply<<<blocks, 256, 0, st>>>(mask, n, region, area, min_area);
  return cudaGetLastError();
}

cudaError_t launch_tissue(const uint16_t* blk8, const SlideGeom& g, int median_k, uint8_t* grey,
                          uint8_t* blurred, int32_t* hist, int32_t* otsu, uint8_t* mask,
                          cudaStream_t st) {
  dim3 g1((g.tw + 127) / 128, g.th);
  k_thumb_grey<<<g1, 128, 0, st>>>(blk8, g.Wp / 8, g.th, g.tw, grey);
  dim3 g2((g.tw + 31) / 32, (g.th + kMedStrip - 1) / kMedStrip);
  k_median<<<g2, 32, 0, st>>>(grey, g.th, g.tw, median_k, blurred);
  cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  long long n = (long long)g.th * g.tw;
  k_hist<<<152, 256, 0, st>>>(blurred, n, hist);
  k_otsu<<<1, 256, 0, st>>>(hist, otsu);
  k_mask<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(blurred, n, otsu, mask);
  return cudaGetLastError();
}

cudaError_t launch_tissue_grey(const uint8_t* grey, const SlideGeom& g, int median_k, uint8_t* blurred,
                               int32_t* hist, int32_t* otsu, uint8_t* mask, cudaStream_t st) {
  dim3 g2((g.tw + 31) / 32, (g.th + kMedStrip - 1) / kMedStrip);
  k_median<<<g2, 32, 0, st>>>(grey, g.th, g.tw, median_k, blurred);
  cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  long long n = (long long)g.th * g.tw;
  k_hist<<<152, 256, 0, st>>>(blurred, n, hist);
  k_otsu<<<1, 256, 0, st>>>(hist, otsu);
  k_mask<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(blurred, n, otsu, mask);
  return cudaGetLastError();
}

cudaError_t launch_tiles(const uint8_t* mask, const SlideGeom& g, int filter, int32_t* tiles,
                         int32_t* counts, uint8_t* flags, int32_t* slot_map, cudaStream_t st) {
  int total = g.grid_off[g.n_scales];
  k_tile_flags<<<(total + 255) / 256, 256, 0, st>>>(mask, g, filter, flags);
  k_tile_compact<<<1, 1024, 0, st>>>(flags, g, tiles, counts, slot_map);
  return cudaGetLastError();
}

}  // namespace omni
