// Backward of the stitched soft-Dice + BCE loss through the dynamic head, the
// controller, the pre-head and the last decoder block (FP32 on the GPU).
//
// Loss (per class c at its scale, over the class's label map of N_c pixels,
// L = stitched logit, g = ground truth, s = sigmoid(L)):
//   dice_c = 1 - (2 I + 1) / (S + G + 1),  I = sum s g, S = sum s, G = sum g
//   bce_c  = mean(max(L, 0) - g L + log(1 + exp(-|L|)))
//   loss   = mean over classes of (dice_c + bce_c)
// dloss/dL = [ -(2 g (S+G+1) - (2 I + 1)) / (S+G+1)^2 * s (1 - s) + (s - g) / N_c ] / n_classes.
// Through the overlap average, a tile's logit at a pixel receives dloss/dL / cov.
// All arithmetic is FP32.  Every reduction is a fixed-order sum (block or
// chunk partials, then one ordered pass), so the gradients are run-to-run
// deterministic; the ordered passes and the gradient accumulators that carry a
// sum across batches are compensated (Kahan 1965: each addition also keeps
// the rounding error it made and feeds it into the next), so their error does
// not grow with the number of terms.  An accumulator is a float2 (sum, carry).
#include "omni_internal.cuh"

namespace omni {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// compensated addition: s + x with the running carry c of the errors so far
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
__device__ __forceinline__ void acc_add(float2* a, float x) {
  float2 v = *a;
  kahan_add(v.x, v.y, x);
  *a = v;
}

template <typename T>
__device__ T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;   // valid in thread 0
}

// partial[blk][4] = (S, I, G, BCE sum) over the block's pixels
__global__ void __launch_bounds__(kRedThreads) k_loss_partial(const float* __restrict__ L,
                                                              const uint8_t* __restrict__ gt, long long n,
                                                              float* __restrict__ partial) {
  __shared__ float sh[32];
  float s = 0, i = 0, g = 0, b = 0, cs = 0, ci = 0, cg = 0, cb = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const float l = L[k];
    const float gg = gt[k] ? 1.f : 0.f;
    const float sg = sigmoidf_(l);
    kahan_add(s, cs, sg);
    kahan_add(i, ci, sg * gg);
    kahan_add(g, cg, gg);
    kahan_add(b, cb, fmaxf(l, 0.f) - gg * l + log1pf(expf(-fabsf(l))));
  }
  float r;
  r = block_sum(s, sh); if (threadIdx.x == 0) partial[blockIdx.x * 4 + 0] = r;
  r = block_sum(i, sh); if (threadIdx.x == 0) partial[blockIdx.x * 4 + 1] = r;
  r = block_sum(g, sh); if (threadIdx.x == 0) partial[blockIdx.x * 4 + 2] = r;
  r = block_sum(b, sh); if (threadIdx.x == 0) partial[blockIdx.x * 4 + 3] = r;
}

// sums[c][4] from the partials of every class (ordered); loss = mean_c(dice + bce)
__global__ void k_loss_final(const float* __restrict__ partial, int blocks, int n_cls, NPix npix,
                             float* __restrict__ sums, float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float total = 0, ct = 0;
  for (int c = 0; c < n_cls; ++c) {
    float a[4] = {0, 0, 0, 0}, ca[4] = {0, 0, 0, 0};
    for (int k = 0; k < blocks; ++k)
      for (int q = 0; q < 4; ++q) kahan_add(a[q], ca[q], partial[((long long)c * blocks + k) * 4 + q]);
    for (int q = 0; q < 4; ++q) sums[c * 4 + q] = a[q];
    const float dice = 1.0f - (2.0f * a[1] + 1.0f) / (a[0] + a[2] + 1.0f);
    kahan_add(total, ct, dice + a[3] / (float)npix.n[c]);
  }
  loss[0] = total / (float)n_cls;
}

__global__ void k_loss_grad(const float* __restrict__ L, const uint8_t* __restrict__ gt, long long n,
                            const float* __restrict__ sums, float npix, int n_cls,
                            float* __restrict__ dL) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float S = sums[0], I = sums[1], G = sums[2];
  const float Bd = S + G + 1.0f, A = 2.0f * I + 1.0f;
  const float l = L[k];
  const float gg = gt[k] ? 1.f : 0.f;
  const float s = sigmoidf_(l);
  const float ddice = -(2.0f * gg * Bd - A) / (Bd * Bd);
  dL[k] = (ddice * s * (1.f - s) + (s - gg) / npix) / (float)n_cls;
}

// a = ReLU(g * c + b) over [n][C]
__global__ void k_affine_relu(const float* __restrict__ c, const float* __restrict__ g,
                              const float* __restrict__ b, int C, long long n, float* __restrict__ a) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n * C) return;
  const int ch = (int)(k % C);
  a[k] = fmaxf(fmaf(g[ch], c[k], b[ch]), 0.f);
}

// da_pre = da * [g1 c1 + b1 > 0]; dc = g1 * da_pre (both [n][C])
__global__ void k_relu_bwd(const float* __restrict__ da, const float* __restrict__ c1,
                           const float* __restrict__ g1, const float* __restrict__ b1, int C, long long n,
                           float* __restrict__ da_pre, float* __restrict__ dc) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n * C) return;
  const int ch = (int)(k % C);
  const float on = fmaf(g1[ch], c1[k], b1[ch]) > 0.f ? 1.f : 0.f;
  const float v = da[k] * on;
  da_pre[k] = v;
  dc[k] = g1[ch] * v;
}

// Head backward for one class of the scale.  Per pixel: recompute
// y0 = ReLU(g2 c2 + b2 + pr), h0 = ReLU(Wh y0 + bh), h1, h2 from theta, take
// dl = dloss/dL / cov at the pixel's label-map position (stitch transpose),
// and accumulate dtheta (153 sums per block) and dh0 (per pixel, summed over
// the classes: overwritten for the first class, added for the others).
constexpr int kHeadBwdThreads = 128;
constexpr int kHeadBwdPix = 8192;

template <int C0>
__global__ void __launch_bounds__(kHeadBwdThreads) k_head_bwd(BwdHeadArgs a) {
  __shared__ float th[kHeadParams];
  __shared__ float wh[kHeadCh * C0], bh[kHeadCh], g2[C0], b2[C0];
  __shared__ float red[kHeadBwdThreads / 32][kHeadParams];
  const int b = blockIdx.y, t = threadIdx.x;
  for (int i = t; i < kHeadParams; i += blockDim.x)
    th[i] = a.theta[((long long)b * a.n_cls + a.ci) * kHeadParams + i];
  for (int i = t; i < kHeadCh * C0; i += blockDim.x) wh[i] = a.wh[i];
  for (int i = t; i < C0; i += blockDim.x) { g2[i] = a.g2[i]; b2[i] = a.b2[i]; }
  if (t < kHeadCh) bh[t] = a.bh[t];
  __syncthreads();
  const long long PP = (long long)a.P * a.P;
  const int ty = a.tiles3[3 * b + 1], tx = a.tiles3[3 * b + 2];
  float acc[kHeadParams];
#pragma unroll
  for (int q = 0; q < kHeadParams; ++q) acc[q] = 0.f;
  const long long p0 = (long long)blockIdx.x * kHeadBwdPix;
  for (int q = t; q < kHeadBwdPix; q += blockDim.x) {
    const long long p = p0 + q;
    if (p >= PP) break;
    const int i = (int)(p / a.P), j = (int)(p % a.P);
    const int oy = ty + i - a.oy0, ox = tx + j - a.ox0;
    float dl = 0.f;
    if (oy >= 0 && oy < a.oh && ox >= 0 && ox < a.ow) {
      const long long o = (long long)oy * a.ow + ox;
      const int cov = a.cov[o];
      if (cov > 0) dl = a.dL[o] / (float)cov;
    }
    const long long px = (long long)b * PP + p;
    float h0[kHeadCh];
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) h0[o] = bh[o];
#pragma unroll
    for (int c = 0; c < C0; ++c) {
      const float y = fmaxf(fmaf(g2[c], a.c2[px * C0 + c], b2[c]) + a.pr[px * C0 + c], 0.f);
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) h0[o] = fmaf(wh[o * C0 + c], y, h0[o]);
    }
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) h0[o] = fmaxf(h0[o], 0.f);
    float h1[kHeadCh], h2[kHeadCh];
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) {
      float s = th[136 + o];
#pragma unroll
      for (int c = 0; c < kHeadCh; ++c) s = fmaf(th[o * 8 + c], h0[c], s);
      h1[o] = fmaxf(s, 0.f);
    }
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) {
      float s = th[144 + o];
#pragma unroll
      for (int c = 0; c < kHeadCh; ++c) s = fmaf(th[64 + o * 8 + c], h1[c], s);
      h2[o] = fmaxf(s, 0.f);
    }
    // logit = W3 h2 + b3
    float dh2[kHeadCh], dh1[kHeadCh], dh0[kHeadCh];
#pragma unroll
    for (int c = 0; c < kHeadCh; ++c) {
      acc[128 + c] += dl * h2[c];                       // dW3
      dh2[c] = h2[c] > 0.f ? dl * th[128 + c] : 0.f;
    }
    acc[152] += dl;                                     // db3
#pragma unroll
    for (int c = 0; c < kHeadCh; ++c) dh1[c] = 0.f;
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) {
      acc[144 + o] += dh2[o];                           // db2
#pragma unroll
      for (int c = 0; c < kHeadCh; ++c) {
        acc[64 + o * 8 + c] += dh2[o] * h1[c];          // dW2
        dh1[c] = fmaf(th[64 + o * 8 + c], dh2[o], dh1[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < kHeadCh; ++c) {
      dh1[c] = h1[c] > 0.f ? dh1[c] : 0.f;
      dh0[c] = 0.f;
    }
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) {
      acc[136 + o] += dh1[o];                           // db1
#pragma unroll
      for (int c = 0; c < kHeadCh; ++c) {
        acc[o * 8 + c] += dh1[o] * h0[c];               // dW1
        dh0[c] = fmaf(th[o * 8 + c], dh1[o], dh0[c]);
      }
    }
    float* d = a.dh0 + px * kHeadCh;
#pragma unroll
    for (int c = 0; c < kHeadCh; ++c) d[c] = a.ci == 0 ? dh0[c] : d[c] + dh0[c];
  }
  // block reduction of the 153 sums (fixed order)
  const int lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int q = 0; q < kHeadParams; ++q) {
    float v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  for (int q = t; q < kHeadParams; q += blockDim.x) {
    float v = 0.f;
    for (int w = 0; w < kHeadBwdThreads / 32; ++w) v += red[w][q];
    a.dtheta_partial[(((long long)b * a.n_cls + a.ci) * gridDim.x + blockIdx.x) * kHeadParams + q] = v;
  }
}

// Pre-head backward: dh0_pre = dh0 * [Wh y0 + bh > 0]; dy0 = Wh^T dh0_pre;
// dy0_pre = dy0 * [y0_pre > 0].  Writes dh0_pre [px][8], y0 [px][C0],
// dy0_pre [px][C0] and dc2 = g2 * dy0_pre [px][C0].
template <int C0>
__global__ void k_prehead_bwd(BwdHeadArgs a, long long npx) {
  __shared__ float wh[kHeadCh * C0], bh[kHeadCh], g2[C0], b2[C0];
  const int t = threadIdx.x;
  for (int i = t; i < kHeadCh * C0; i += blockDim.x) wh[i] = a.wh[i];
  for (int i = t; i < C0; i += blockDim.x) { g2[i] = a.g2[i]; b2[i] = a.b2[i]; }
  if (t < kHeadCh) bh[t] = a.bh[t];
  __syncthreads();
  const long long px = blockIdx.x * (long long)blockDim.x + t;
  if (px >= npx) return;
  float ypre[C0], y[C0];
  float h[kHeadCh];
#pragma unroll
  for (int o = 0; o < kHeadCh; ++o) h[o] = bh[o];
#pragma unroll
  for (int c = 0; c < C0; ++c) {
    ypre[c] = fmaf(g2[c], a.c2[px * C0 + c], b2[c]) + a.pr[px * C0 + c];
    y[c] = fmaxf(ypre[c], 0.f);
    a.y0[px * C0 + c] = y[c];
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) h[o] = fmaf(wh[o * C0 + c], y[c], h[o]);
  }
  float dpre[kHeadCh];
#pragma unroll
  for (int o = 0; o < kHeadCh; ++o) {
    dpre[o] = h[o] > 0.f ? a.dh0[px * kHeadCh + o] : 0.f;
    a.dh0_pre[px * kHeadCh + o] = dpre[o];
  }
#pragma unroll
  for (int c = 0; c < C0; ++c) {
    float d = 0.f;
#pragma unroll
    for (int o = 0; o < kHeadCh; ++o) d = fmaf(wh[o * C0 + c], dpre[o], d);
    d = ypre[c] > 0.f ? d : 0.f;
    a.dy0_pre[px * C0 + c] = d;
    a.dc2[px * C0 + c] = g2[c] * d;
  }
}

// partial[chunk][o][k] = sum over the chunk's pixels of dY[px][o] * X(px, k),
// X(px, k) = input channel (k % cin) at the pixel shifted by tap (k / cin)
// (9 taps of a zero-padded 3x3 window, or the centre only), within its tile.
constexpr int kWgThreads = 256;
constexpr int kWgChunk = 8192;
template <int O>
__global__ void __launch_bounds__(kWgThreads) k_wgrad(const float* __restrict__ dY,
                                                      const float* __restrict__ X, int x_cs, int cin,
                                                      int taps, int P, long long npx,
                                                      float* __restrict__ partial, int K) {
  __shared__ __align__(16) float sy[32][O];
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  const int tap = taps == 9 ? k / cin : 4, c = k % cin;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  float acc[O];
#pragma unroll
  for (int o = 0; o < O; ++o) acc[o] = 0.f;
  const long long pbeg = (long long)blockIdx.x * kWgChunk;
  const long long PP = (long long)P * P;
  for (long long p0 = pbeg; p0 < pbeg + kWgChunk && p0 < npx; p0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * O; e += blockDim.x) {
      const int r = e / O, o = e % O;
      const long long px = p0 + r;
      sy[r][o] = px < npx ? dY[px * O + o] : 0.f;
    }
    __syncthreads();
    if (k < K) {
      for (int r = 0; r < 32; ++r) {
        const long long px = p0 + r;
        if (px >= npx) break;
        const long long b = px / PP;
        const int rem = (int)(px - b * PP);
        const int i = rem / P + dy, j = rem % P + dx;
        float x = 0.f;
        if (i >= 0 && i < P && j >= 0 && j < P) x = X[(b * PP + (long long)i * P + j) * x_cs + c];
        const float4* yr = reinterpret_cast<const float4*>(sy[r]);
#pragma unroll
        for (int o4 = 0; o4 < O / 4; ++o4) {
          const float4 v = yr[o4];
          acc[o4 * 4 + 0] = fmaf(v.x, x, acc[o4 * 4 + 0]);
          acc[o4 * 4 + 1] = fmaf(v.y, x, acc[o4 * 4 + 1]);
          acc[o4 * 4 + 2] = fmaf(v.z, x, acc[o4 * 4 + 2]);
          acc[o4 * 4 + 3] = fmaf(v.w, x, acc[o4 * 4 + 3]);
        }
      }
    }
  }
  if (k < K) {
#pragma unroll
    for (int o = 0; o < O; ++o) partial[((long long)blockIdx.x * O + o) * K + k] = acc[o];
  }
}

// partial[chunk][c] = sum over the chunk of A[px][c] (* B[px][c] when B != null)
__global__ void k_colsum(const float* __restrict__ A, const float* __restrict__ B, int C, long long npx,
                         float* __restrict__ partial) {
  const int c = threadIdx.x;
  if (c >= C) return;
  const long long pbeg = (long long)blockIdx.x * kWgChunk;
  float s = 0.f;
  for (long long px = pbeg; px < pbeg + kWgChunk && px < npx; ++px)
    s += B ? A[px * C + c] * B[px * C + c] : A[px * C + c];
  partial[(long long)blockIdx.x * C + c] = s;
}

// acc[i] += sum over chunks (in order) of partial[chunk][i], both compensated
__global__ void k_reduce(const float* __restrict__ partial, int chunks, long long n, float2* __restrict__ acc) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0, c = 0;
  for (int k = 0; k < chunks; ++k) kahan_add(s, c, partial[(long long)k * n + i]);
  acc_add(acc + i, s);
}

// Controller backward for a batch: dWc[row][k] += sum_{b, ci} dtheta[b][ci][row] z_{b,ci}[k],
// dbc[row] += sum dtheta, with z = [g_b; onehot(class); onehot(scale)].
__global__ void k_ctrl_bwd(const float* __restrict__ dtheta_partial, int hblocks, int B, int n_cls,
                           const int* __restrict__ cls_ids, int n_classes, int n_scales, int scale,
                           const float* __restrict__ g, int Cb, float2* __restrict__ dwc,
                           float2* __restrict__ dbc) {
  const int row = blockIdx.x;
  const int zdim = Cb + n_classes + n_scales;
  __shared__ float dt[64][OMNI_MAX_CLASSES];
  for (int e = threadIdx.x; e < B * n_cls; e += blockDim.x) {
    const int b = e / n_cls, ci = e % n_cls;
    float s = 0, c = 0;
    for (int k = 0; k < hblocks; ++k)
      kahan_add(s, c, dtheta_partial[(((long long)b * n_cls + ci) * hblocks + k) * kHeadParams + row]);
    dt[b][ci] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < zdim; k += blockDim.x) {
    float s = 0, c = 0;
    for (int b = 0; b < B; ++b)
      for (int ci = 0; ci < n_cls; ++ci) {
        float z = 0;
        if (k < Cb) z = g[(long long)b * Cb + k];
        else if (k == Cb + cls_ids[ci]) z = 1.0f;
        else if (k == Cb + n_classes + scale) z = 1.0f;
        kahan_add(s, c, dt[b][ci] * z);
      }
    acc_add(dwc + (long long)row * zdim + k, s);
  }
  if (threadIdx.x == 0) {
    float s = 0, c = 0;
    for (int b = 0; b < B; ++b)
      for (int ci = 0; ci < n_cls; ++ci) kahan_add(s, c, dt[b][ci]);
    acc_add(dbc + row, s);
  }
}

// accumulator (sum, carry) -> FP32 value: the carry holds the negated error
// of the last additions
__global__ void k_to_f32(const float2* __restrict__ a, long long n, float* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i].x - a[i].y;
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int loss_blocks() { return 256; }

cudaError_t launch_loss_partial(const float* L, const uint8_t* gt, long long n, float* partial,
                                cudaStream_t st) {
  k_loss_partial<<<loss_blocks(), kRedThreads, 0, st>>>(L, gt, n, partial);
  return cudaGetLastError();
}
cudaError_t launch_loss_final(const float* partial, int n_cls, const NPix& npix, float* sums,
                              float* loss, cudaStream_t st) {
  k_loss_final<<<1, 32, 0, st>>>(partial, loss_blocks(), n_cls, npix, sums, loss);
  return cudaGetLastError();
}
cudaError_t launch_loss_grad(const float* L, const uint8_t* gt, long long n, const float* sums, float npix,
                             int n_cls, float* dL, cudaStream_t st) {
  k_loss_grad<<<blocks_for(n, 256), 256, 0, st>>>(L, gt, n, sums, npix, n_cls, dL);
  return cudaGetLastError();
}
cudaError_t launch_affine_relu(const float* c, const float* g, const float* b, int C, long long n, float* a,
                               cudaStream_t st) {
  k_affine_relu<<<blocks_for(n * C, 256), 256, 0, st>>>(c, g, b, C, n, a);
  return cudaGetLastError();
}
cudaError_t launch_relu_bwd(const float* da, const float* c1, const float* g1, const float* b1, int C, long long n,
                            float* da_pre, float* dc, cudaStream_t st) {
  k_relu_bwd<<<blocks_for(n * C, 256), 256, 0, st>>>(da, c1, g1, b1, C, n, da_pre, dc);
  return cudaGetLastError();
}
int head_bwd_blocks(int P) { return (int)(((long long)P * P + kHeadBwdPix - 1) / kHeadBwdPix); }
cudaError_t launch_head_bwd(const BwdHeadArgs& a, int C0, cudaStream_t st) {
  dim3 grid(head_bwd_blocks(a.P), a.B);
  switch (C0) {
    case 8: k_head_bwd<8><<<grid, kHeadBwdThreads, 0, st>>>(a); break;
    case 16: k_head_bwd<16><<<grid, kHeadBwdThreads, 0, st>>>(a); break;
    case 32: k_head_bwd<32><<<grid, kHeadBwdThreads, 0, st>>>(a); break;
    case 64: k_head_bwd<64><<<grid, kHeadBwdThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
cudaError_t launch_prehead_bwd(const BwdHeadArgs& a, int C0, long long npx, cudaStream_t st) {
  const unsigned g = blocks_for(npx, 128);
  switch (C0) {
    case 8: k_prehead_bwd<8><<<g, 128, 0, st>>>(a, npx); break;
    case 16: k_prehead_bwd<16><<<g, 128, 0, st>>>(a, npx); break;
    case 32: k_prehead_bwd<32><<<g, 128, 0, st>>>(a, npx); break;
    case 64: k_prehead_bwd<64><<<g, 128, 0, st>>>(a, npx); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
int wgrad_chunks(long long npx) { return (int)((npx + kWgChunk - 1) / kWgChunk); }
cudaError_t launch_wgrad(const float* dY, int O, const float* X, int x_cs, int cin, int taps, int P,
                         long long npx, float* partial, float2* acc, cudaStream_t st) {
  if (O > 64 || O % 4) return cudaErrorInvalidValue;
  const int K = taps * cin;
  const int chunks = wgrad_chunks(npx);
  dim3 grid(chunks, (K + kWgThreads - 1) / kWgThreads);
  switch (O) {
    case 8: k_wgrad<8><<<grid, kWgThreads, 0, st>>>(dY, X, x_cs, cin, taps, P, npx, partial, K); break;
    case 16: k_wgrad<16><<<grid, kWgThreads, 0, st>>>(dY, X, x_cs, cin, taps, P, npx, partial, K); break;
    case 32: k_wgrad<32><<<grid, kWgThreads, 0, st>>>(dY, X, x_cs, cin, taps, P, npx, partial, K); break;
    case 64: k_wgrad<64><<<grid, kWgThreads, 0, st>>>(dY, X, x_cs, cin, taps, P, npx, partial, K); break;
    default: return cudaErrorInvalidValue;
  }
  const long long n = (long long)O * K;
  k_reduce<<<blocks_for(n, 256), 256, 0, st>>>(partial, chunks, n, acc);
  return cudaGetLastError();
}
cudaError_t launch_colsum(const float* A, const float* B, int C, long long npx, float* partial, float2* acc,
                          cudaStream_t st) {
  if (C > 1024) return cudaErrorInvalidValue;
  const int chunks = wgrad_chunks(npx);
  k_colsum<<<chunks, ((C + 31) / 32) * 32, 0, st>>>(A, B, C, npx, partial);
  k_reduce<<<blocks_for(C, 256), 256, 0, st>>>(partial, chunks, C, acc);
  return cudaGetLastError();
}
cudaError_t launch_ctrl_bwd(const float* dtheta_partial, int hblocks, int B, int n_cls, const int* cls_ids_dev,
                            int n_classes, int n_scales, int scale, const float* g, int Cb, float2* dwc,
                            float2* dbc, cudaStream_t st) {
  if (B > 64) return cudaErrorInvalidValue;
  k_ctrl_bwd<<<kHeadParams, 256, 0, st>>>(dtheta_partial, hblocks, B, n_cls, cls_ids_dev, n_classes, n_scales,
                                          scale, g, Cb, dwc, dbc);
  return cudaGetLastError();
}
cudaError_t launch_to_f32(const float2* a, long long n, float* out, cudaStream_t st) {
  k_to_f32<<<blocks_for(n, 256), 256, 0, st>>>(a, n, out);
  return cudaGetLastError();
}

}  // namespace omni
