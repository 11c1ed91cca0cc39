// Omni-Seg dynamic head (Sec. 2.2): a controller turns the tile's global
// average-pooled bottleneck feature plus one-hot class and scale codes into the
// 153 parameters of a per-tile, per-class 1x1 head 8 -> 8 -> 8 -> 1, which is
// applied at every pixel of the pre-head feature h0 = ReLU(Wh y0 + bh).
//
// Two kernels: k_controller evaluates theta for every tile of a batch and every
// class of the scale (the controller weights are read once per batch, not once
// per pixel block), and k_head runs the pre-head and all heads of the scale
// over the tile pixels, writing FP32 logits.
#include <cuda_fp16.h>

#include "omni_internal.cuh"

namespace omni {
namespace {

constexpr int kHeadThreads = 128;
constexpr int kPixPerBlock = 4096;
constexpr int kCtrlRows = 32;          // controller rows per block

// grid = (ceil(153 / kCtrlRows), tiles); block = 8 warps, one theta row per warp step
__global__ void __launch_bounds__(256) k_controller(HeadArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int zdim = a.Cb + a.n_classes + a.n_scales;
  const int r0 = blockIdx.x * kCtrlRows, b = blockIdx.y;
  for (int q = warp; q < kCtrlRows; q += 8) {
    const int row = r0 + q;
    if (row >= kHeadParams) continue;
    const float* w = a.wc + (long long)row * zdim;
    const float* g = a.g + (long long)b * a.Cb;
    float s = 0.f;
    for (int k = lane; k < a.Cb; k += 32) s = fmaf(w[k], g[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane < a.n_cls_here) {
      const float th = s + w[a.Cb + a.n_classes + a.scale] + a.bc[row] + w[a.Cb + a.cls_ids[lane]];
      a.theta[((long long)b * a.n_cls_here + lane) * kHeadParams + row] = th;
    }
  }
}

template <typename T> struct Load8;
template <> struct Load8<float> {
  static __device__ __forceinline__ void f(const float* p, float v[8]) {
    const float4 x = *reinterpret_cast<const float4*>(p), y = *reinterpret_cast<const float4*>(p + 4);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w; v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  }
};
template <> struct Load8<__nv_bfloat16> {
  static __device__ __forceinline__ void f(const __nv_bfloat16* p, float v[8]) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
};

template <> struct Load8<__half> {
  static __device__ __forceinline__ void f(const __half* p, float v[8]) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
};

// Each thread evaluates kHeadPx pixels (kHeadThreads apart, so a warp's loads
// cover consecutive pixels) and reuses every weight it reads from shared
// memory for all of them; theta rows are padded to 160 floats so they are
// 16-byte aligned for vector loads.
constexpr int kHeadPx = 4;
constexpr int kThetaStride = 160;

template <int C0, typename T>
__global__ void __launch_bounds__(kHeadThreads) k_head(HeadArgs a) {
  __shared__ __align__(16) float theta[OMNI_MAX_CLASSES][kThetaStride];
  __shared__ __align__(16) float wh[kHeadCh * C0];
  __shared__ float bh[kHeadCh];
  const int b = blockIdx.y;
  const int t = threadIdx.x;
  for (int i = t; i < kHeadCh * C0; i += kHeadThreads) wh[i] = a.wh[i];
  if (t < kHeadCh) bh[t] = a.bh[t];
  for (int i = t; i < a.n_cls_here * kHeadParams; i += kHeadThreads)
    theta[i / kHeadParams][i % kHeadParams] = a.theta[(long long)b * a.n_cls_here * kHeadParams + i];
  __syncthreads();

  const long long PP = (long long)a.P * a.P;
  const T* Y = static_cast<const T*>(a.y0) + (long long)b * PP * C0;
  float* out = a.logits + (long long)(a.slot0 + b) * a.n_cls_here * PP;
  const long long p0 = (long long)blockIdx.x * kPixPerBlock;
  for (int q0 = 0; q0 < kPixPerBlock; q0 += kHeadThreads * kHeadPx) {
    long long pix[kHeadPx];
    bool live[kHeadPx];
#pragma unroll
    for (int u = 0; u < kHeadPx; ++u) {
      pix[u] = p0 + q0 + u * kHeadThreads + t;
      live[u] = pix[u] < PP;
    }
    if (!live[0]) break;
    float h0[kHeadPx][kHeadCh];
#pragma unroll
    for (int u = 0; u < kHeadPx; ++u)
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) h0[u][o] = bh[o];
#pragma unroll
    for (int c0 = 0; c0 < C0; c0 += 8) {
      float y[kHeadPx][8];
#pragma unroll
      for (int u = 0; u < kHeadPx; ++u) {
        if (live[u]) Load8<T>::f(Y + pix[u] * C0 + c0, y[u]);
        else
#pragma unroll
          for (int c = 0; c < 8; ++c) y[u][c] = 0.f;
      }
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) {
        const float4 w0 = *reinterpret_cast<const float4*>(&wh[o * C0 + c0]);
        const float4 w1 = *reinterpret_cast<const float4*>(&wh[o * C0 + c0 + 4]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
          for (int u = 0; u < kHeadPx; ++u) h0[u][o] = fmaf(w[c], y[u][c], h0[u][o]);
      }
    }
#pragma unroll
    for (int u = 0; u < kHeadPx; ++u)
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) h0[u][o] = fmaxf(h0[u][o], 0.f);
    for (int ci = 0; ci < a.n_cls_here; ++ci) {
      const float* th = theta[ci];
      float h1[kHeadPx][kHeadCh], h2[kHeadPx][kHeadCh];
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) {
        const float4 w0 = *reinterpret_cast<const float4*>(&th[o * 8]);
        const float4 w1 = *reinterpret_cast<const float4*>(&th[o * 8 + 4]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const float bias = th[136 + o];
#pragma unroll
        for (int u = 0; u < kHeadPx; ++u) {
          float s = bias;
#pragma unroll
          for (int c = 0; c < kHeadCh; ++c) s = fmaf(w[c], h0[u][c], s);
          h1[u][o] = fmaxf(s, 0.f);
        }
      }
#pragma unroll
      for (int o = 0; o < kHeadCh; ++o) {
        const float4 w0 = *reinterpret_cast<const float4*>(&th[64 + o * 8]);
        const float4 w1 = *reinterpret_cast<const float4*>(&th[64 + o * 8 + 4]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const float bias = th[144 + o];
#pragma unroll
        for (int u = 0; u < kHeadPx; ++u) {
          float s = bias;
#pragma unroll
          for (int c = 0; c < kHeadCh; ++c) s = fmaf(w[c], h1[u][c], s);
          h2[u][o] = fmaxf(s, 0.f);
        }
      }
      const float4 w0 = *reinterpret_cast<const float4*>(&th[128]);
      const float4 w1 = *reinterpret_cast<const float4*>(&th[132]);
      const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
      for (int u = 0; u < kHeadPx; ++u) {
        float s = th[152];
#pragma unroll
        for (int c = 0; c < kHeadCh; ++c) s = fmaf(w[c], h2[u][c], s);
        if (live[u]) out[ci * PP + pix[u]] = s;
      }
    }
  }
}

template <typename T>
cudaError_t head_t(const HeadArgs& a, cudaStream_t st) {
  long long PP = (long long)a.P * a.P;
  dim3 grid((unsigned)((PP + kPixPerBlock - 1) / kPixPerBlock), a.B);
  switch (a.C0) {
    case 8: k_head<8, T><<<grid, kHeadThreads, 0, st>>>(a); break;
    case 16: k_head<16, T><<<grid, kHeadThreads, 0, st>>>(a); break;
    case 32: k_head<32, T><<<grid, kHeadThreads, 0, st>>>(a); break;
    case 64: k_head<64, T><<<grid, kHeadThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_controller(const HeadArgs& a, cudaStream_t st) {
  if (a.n_cls_here < 1 || a.n_cls_here > OMNI_MAX_CLASSES) return cudaErrorInvalidValue;
  if (a.B < 1) return cudaErrorInvalidValue;
  k_controller<<<dim3((kHeadParams + kCtrlRows - 1) / kCtrlRows, a.B), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_head(const HeadArgs& a, cudaStream_t st) {
  if (a.n_cls_here < 1 || a.n_cls_here > OMNI_MAX_CLASSES) return cudaErrorInvalidValue;
  if (a.precision == OMNI_FP32) return head_t<float>(a, st);
  return a.precision == OMNI_FP16 ? head_t<__half>(a, st) : head_t<__nv_bfloat16>(a, st);
}

}  // namespace omni
