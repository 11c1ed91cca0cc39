// Residual U-Net building blocks on the CUDA cores (the plain FP32 path),
// plus the precision-generic pieces both paths share: the first convolution
// (reads the uint8 tile straight from the canvas), 2x2 max-pool, bilinear x2
// upsampling into the decoder's concat buffer, and global average pooling.
//
// Block structure (residual U-Net of the Omni-Seg network, Sec. 2.2):
//   out = ReLU(g2 * conv3x3(ReLU(g1 * conv3x3(x) + b1)) + b2 + wp . x)
// The SIMT implicit GEMM below computes one such convolution with the norm,
// the 1x1 residual projection and the ReLU fused into its epilogue.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "omni_internal.cuh"

namespace omni {
namespace {

template <typename T> struct Vec8;
template <> struct Vec8<float> {
  static __device__ __forceinline__ void load(const float* p, float v[8]) {
    float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  static __device__ __forceinline__ void store(float* p, const float v[8]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
  }
};
template <> struct Vec8<__nv_bfloat16> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* p, float v[8]) {
    uint4 q = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __bfloat1622float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
  static __device__ __forceinline__ void store(__nv_bfloat16* p, const float v[8]) {
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(p) = q;
  }
};

template <> struct Vec8<__half> {
  static __device__ __forceinline__ void load(const __half* p, float v[8]) {
    uint4 q = *reinterpret_cast<const uint4*>(p);
    const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 f = __half22float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
  static __device__ __forceinline__ void store(__half* p, const float v[8]) {
    uint4 q;
    __half2* h = reinterpret_cast<__half2*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(p) = q;
  }
};

// v = 2 u / 255 - 1  (input normalisation of the tile)
__device__ __forceinline__ float norm_u8(uint8_t u) { return 2.0f * (float)u / 255.0f - 1.0f; }

// ------------------------------------------------------------------ first conv
// conv3x3 over the 3 normalised colour channels of a tile read in place from
// the uint8 canvas (zero padding at the tile border), norm, ReLU.
// Each thread computes four horizontally adjacent pixels so every weight read
// from shared memory feeds four FMAs.  grid: x = column quads, y = row, z = tile.
constexpr int kFirstPix = 4;
template <int C0, typename T>
__global__ void __launch_bounds__(128) k_conv_first(int P, const CanvasTab cv,
                                                    const int32_t* __restrict__ tiles3,
                                                    const float* __restrict__ w27,  // [27][C0]
                                                    const float* __restrict__ gamma,
                                                    const float* __restrict__ beta,
                                                    T* __restrict__ y, int y_cs, int y_co) {
  __shared__ float ws[27 * C0];
  __shared__ float gs[C0], bs[C0];
  for (int i = threadIdx.x; i < 27 * C0; i += blockDim.x) ws[i] = w27[i];
  for (int i = threadIdx.x; i < C0; i += blockDim.x) { gs[i] = gamma[i]; bs[i] = beta[i]; }
  __syncthreads();
  const int j0 = (blockIdx.x * blockDim.x + threadIdx.x) * kFirstPix;
  if (j0 >= P) return;
  const int i = blockIdx.y, b = blockIdx.z;
  const int ty = tiles3[3 * b + 1], tx = tiles3[3 * b + 2];
  const uint8_t* __restrict__ canvas = cv.ptr[tiles3[3 * b]];
  const long long cstride = cv.stride[tiles3[3 * b]];
  // 3 rows x 6 columns x 3 channels of normalised input around the four pixels
  float in[3][kFirstPix + 2][3];
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int q = 0; q < kFirstPix + 2; ++q) {
      const int ii = i + dy - 1, jj = j0 + q - 1;
      const bool ok = ii >= 0 && ii < P && jj >= 0 && jj < P;
      // address of a pixel inside the tile even where the window leaves it
      const int ic = min(max(ii, 0), P - 1), jc = min(max(jj, 0), P - 1);
      const uint8_t* p = canvas + (long long)(ty + ic) * cstride + (long long)(tx + jc) * 3;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = norm_u8(p[c]);
        in[dy][q][c] = ok ? v : 0.0f;
      }
    }
  T* out = y + (((long long)b * P + i) * P + j0) * y_cs + y_co;
#pragma unroll 1
  for (int o0 = 0; o0 < C0; o0 += 8) {
    float acc[kFirstPix][8];
#pragma unroll
    for (int u = 0; u < kFirstPix; ++u)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[u][q] = 0.0f;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float* wr = ws + ((dy * 3 + dx) * 3 + c) * C0 + o0;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float w = wr[q];
#pragma unroll
            for (int u = 0; u < kFirstPix; ++u) acc[u][q] = fmaf(in[dy][u + dx][c], w, acc[u][q]);
          }
        }
#pragma unroll
    for (int u = 0; u < kFirstPix; ++u) {
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[u][q] = fmaxf(fmaf(gs[o0 + q], acc[u][q], bs[o0 + q]), 0.0f);
      Vec8<T>::store(out + (long long)u * y_cs + o0, acc[u]);
    }
  }
}

// ------------------------------------------------------------------ FP32 implicit GEMM conv
// GEMM view: M = B*R*R output pixels, N = cout, K = 9*cin (tap-major, then
// channel).  Block tile 128 x BN, K step 8, 256 threads, each thread a
// TM x 4 register tile; A is gathered from the shifted NHWC input with zero
// padding, B is the K-major weight matrix.  A second K loop over the 1x1
// residual projection accumulates separately so the epilogue can apply
// ReLU(g * acc + b + acc_res).
constexpr int kBM = 128, kBK = 8, kThreads = 256;

template <int BN>
__global__ void __launch_bounds__(kThreads) k_conv_f32(ConvArgs a) {
  constexpr int TN = 4;
  constexpr int NT = BN / TN;            // threads along N
  constexpr int MT = kThreads / NT;      // threads along M
  constexpr int TM = kBM / MT;
  __shared__ __align__(16) float As[2][kBK][kBM];
  __shared__ __align__(16) float Bs[2][kBK][BN];

  const int t = threadIdx.x;
  const int tn = t % NT, tm = t / NT;
  const long long M = (long long)a.B * a.R * a.R;
  const long long m0 = (long long)blockIdx.x * kBM;
  const int n0 = blockIdx.y * BN;
  const int RR = a.R * a.R;
  const float* X = static_cast<const float*>(a.x);
  const float* Rin = static_cast<const float*>(a.r);

  // this thread's A-load pixel (one float4 of 4 channels per stage)
  const int lm = t >> 1, lc = (t & 1) * 4;
  const long long gm = m0 + lm;
  const bool mvalid = gm < M;
  int lb = 0, li = 0, lj = 0;
  if (mvalid) {
    lb = (int)(gm / RR);
    int rem = (int)(gm - (long long)lb * RR);
    li = rem / a.R;
    lj = rem % a.R;
  }
  // B-load: 8 x BN floats = 2*BN float4
  const int bk = t / (BN / 4), bn = (t % (BN / 4)) * 4;
  const bool bload = t < 2 * BN;

  const int nk_main = 9 * (a.cin / kBK);
  const int nk_res = a.res_mode == RES_TENSOR ? a.cr / kBK : 0;
  const int nk = nk_main + nk_res;

  auto loadA = [&](int kt) -> float4 {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!mvalid) return v;
    if (kt < nk_main) {
      int tap = kt / (a.cin / kBK);
      int c0 = (kt % (a.cin / kBK)) * kBK + lc;
      int ii = li + tap / 3 - 1, jj = lj + tap % 3 - 1;
      if (ii >= 0 && ii < a.R && jj >= 0 && jj < a.R)
        v = *reinterpret_cast<const float4*>(
            X + ((long long)lb * RR + (long long)ii * a.R + jj) * a.x_cs + a.x_co + c0);
    } else {
      int c0 = (kt - nk_main) * kBK + lc;
      v = *reinterpret_cast<const float4*>(Rin + gm * a.r_cs + a.r_co + c0);
    }
    return v;
  };
  auto loadB = [&](int kt) -> float4 {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!bload) return v;
    const float* W = kt < nk_main ? a.w.w_f32 + (long long)(kt * kBK + bk) * a.cout
                                  : a.w.wp_f32 + (long long)((kt - nk_main) * kBK + bk) * a.cout;
    return *reinterpret_cast<const float4*>(W + n0 + bn);
  };
  auto storeA = [&](int buf, float4 v) {
    As[buf][lc + 0][lm] = v.x;
    As[buf][lc + 1][lm] = v.y;
    As[buf][lc + 2][lm] = v.z;
    As[buf][lc + 3][lm] = v.w;
  };
  auto storeB = [&](int buf, float4 v) {
    if (bload) *reinterpret_cast<float4*>(&Bs[buf][bk][bn]) = v;
  };

  float acc[TM][TN], accr[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) { acc[i][j] = 0.f; accr[i][j] = 0.f; }

  float4 ra = loadA(0), rb = loadB(0);
  storeA(0, ra);
  storeB(0, rb);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) { ra = loadA(kt + 1); rb = loadB(kt + 1); }
    const bool res = kt >= nk_main;
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[cur][kk][tm * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[cur][kk][tn * TN + j];
      if (!res) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      } else {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) accr[i][j] = fmaf(av[i], bv[j], accr[i][j]);
      }
    }
    if (kt + 1 < nk) {
      storeA(cur ^ 1, ra);
      storeB(cur ^ 1, rb);
    }
    __syncthreads();
  }

  // epilogue
  float g[TN], be[TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    g[j] = a.w.gamma[n0 + tn * TN + j];
    be[j] = a.w.beta[n0 + tn * TN + j];
  }
  float* Y = static_cast<float*>(a.y);
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    long long m = m0 + tm * TM + i;
    if (m >= M) continue;
    float o[TN];
    if (a.res_mode == RES_RGB) {
      int b = (int)(m / RR);
      int rem = (int)(m - (long long)b * RR);
      int pi = rem / a.R, pj = rem % a.R;
      const int sl = a.tiles3[3 * b];
      const uint8_t* px = a.cv.ptr[sl] + (long long)(a.tiles3[3 * b + 1] + pi) * a.cv.stride[sl] +
                          (long long)(a.tiles3[3 * b + 2] + pj) * 3;
      float v0 = norm_u8(px[0]), v1 = norm_u8(px[1]), v2 = norm_u8(px[2]);
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int n = n0 + tn * TN + j;
        accr[i][j] = fmaf(v0, a.w.wp_f32[n],
                          fmaf(v1, a.w.wp_f32[a.cout + n], v2 * a.w.wp_f32[2 * a.cout + n]));
      }
    }
    if (a.raw) {
      *reinterpret_cast<float4*>(Y + m * a.y_cs + a.y_co + n0 + tn * TN) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      if (a.res_mode == RES_TENSOR)
        *reinterpret_cast<float4*>(static_cast<float*>(a.y2) + m * a.y2_cs + n0 + tn * TN) =
            make_float4(accr[i][0], accr[i][1], accr[i][2], accr[i][3]);
      continue;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) o[j] = fmaxf(fmaf(g[j], acc[i][j], be[j]) + accr[i][j], 0.f);
    *reinterpret_cast<float4*>(Y + m * a.y_cs + a.y_co + n0 + tn * TN) =
        make_float4(o[0], o[1], o[2], o[3]);
  }
}

// ------------------------------------------------------------------ pooling / upsampling
// grid: x = (output column, 8-channel group), y = output row, z = image
template <typename T>
__global__ void k_maxpool(int R, int C, const T* __restrict__ x, int x_cs, int x_co,
                          T* __restrict__ y, int y_cs, int y_co) {
  const int Ro = R >> 1, cg = C >> 3;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Ro * cg) return;
  const int j = t / cg, c = (t - j * cg) * 8;
  const int i = blockIdx.y, b = blockIdx.z;
  float m[8], v[8];
  const T* base = x + ((long long)b * R * R) * x_cs + x_co + c;
  Vec8<T>::load(base + ((long long)(2 * i) * R + 2 * j) * x_cs, m);
  const int offs[3][2] = {{0, 1}, {1, 0}, {1, 1}};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    Vec8<T>::load(base + ((long long)(2 * i + offs[q][0]) * R + 2 * j + offs[q][1]) * x_cs, v);
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = fmaxf(m[k], v[k]);
  }
  Vec8<T>::store(y + (((long long)b * Ro + i) * Ro + j) * y_cs + y_co + c, m);
}

// bilinear x2, half-pixel centres (align_corners = False), edge clamp.
// Output rows (and columns) come in pairs (2k+1, 2k+2) that depend on input
// rows k and k+1 only: row 2k+1 = 0.75 in(k) + 0.25 in(k+1), row 2k+2 =
// 0.25 in(k) + 0.75 in(k+1), k = -1 .. Ri-1, input indices clamped to the
// image (so row 0 = in(0) and row 2Ri-1 = in(Ri-1)); the same in x.  A thread
// owns one output row pair, 8 channels and kUpSeg column pairs: it walks
// along x carrying the previous input column, so each step loads one new
// input column (two rows) and writes a 2 x 2 output block.
// grid: x = (column segment, channel group), y = row pair k + 1, z = tile.
constexpr int kUpSeg = 8;
template <typename T>
__global__ void __launch_bounds__(128) k_upsample(int Ri, int C, const T* __restrict__ x, int x_cs, int x_co,
                                                  T* __restrict__ y, int y_cs, int y_co) {
  const int cg = C >> 3, R = 2 * Ri;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nseg = (Ri + 1 + kUpSeg - 1) / kUpSeg;
  if (t >= nseg * cg) return;
  const int seg = t / cg, c = (t - seg * cg) * 8;
  const int k = (int)blockIdx.y - 1, b = blockIdx.z;
  const int ka = max(k, 0), kb = min(k + 1, Ri - 1);
  const T* xa = x + ((long long)b * Ri + ka) * Ri * x_cs + x_co + c;
  const T* xb = x + ((long long)b * Ri + kb) * Ri * x_cs + x_co + c;
  T* y0 = y + ((long long)b * R + (2 * k + 1)) * R * y_cs + y_co + c;   // row 2k+1
  T* y1 = y0 + (long long)R * y_cs;                                      // row 2k+2
  const bool w0 = k >= 0, w1 = k + 1 < Ri;
  const int l_beg = seg * kUpSeg - 1, l_end = min(l_beg + kUpSeg, Ri);   // column pairs l_beg .. l_end-1
  float pa[8], pb[8], ca[8], cb[8], top0[8], bot0[8];
  Vec8<T>::load(xa + (long long)max(l_beg, 0) * x_cs, pa);
  Vec8<T>::load(xb + (long long)max(l_beg, 0) * x_cs, pb);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    top0[q] = 0.75f * pa[q] + 0.25f * pb[q];
    bot0[q] = 0.25f * pa[q] + 0.75f * pb[q];
  }
  // unrolled: the next columns' loads issue before this column's stores
#pragma unroll 4
  for (int l = l_beg; l < l_end; ++l) {
    const int ln = min(l + 1, Ri - 1);
    Vec8<T>::load(xa + (long long)ln * x_cs, ca);
    Vec8<T>::load(xb + (long long)ln * x_cs, cb);
    float top1[8], bot1[8], o[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      top1[q] = 0.75f * ca[q] + 0.25f * cb[q];
      bot1[q] = 0.25f * ca[q] + 0.75f * cb[q];
    }
    const int j0 = 2 * l + 1, j1 = 2 * l + 2;       // output columns of this pair
    if (w0) {
      if (l >= 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = 0.75f * top0[q] + 0.25f * top1[q];
        Vec8<T>::store(y0 + (long long)j0 * y_cs, o);
      }
      if (j1 < R) {
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = 0.25f * top0[q] + 0.75f * top1[q];
        Vec8<T>::store(y0 + (long long)j1 * y_cs, o);
      }
    }
    if (w1) {
      if (l >= 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = 0.75f * bot0[q] + 0.25f * bot1[q];
        Vec8<T>::store(y1 + (long long)j0 * y_cs, o);
      }
      if (j1 < R) {
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = 0.25f * bot0[q] + 0.75f * bot1[q];
        Vec8<T>::store(y1 + (long long)j1 * y_cs, o);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      top0[q] = top1[q];
      bot0[q] = bot1[q];
    }
  }
}

// g[b][c] = mean over the R x R pixels of tile b.  Block (b, 32-channel group):
// 8 pixel phases x 32 channels; phase h sums pixels h, h+8, ... in order, then
// the 8 phase sums are added in phase order (a fixed summation order).
template <int C0, typename T>
cudaError_t first_t(const ConvArgs& a, cudaStream_t st) {
  if (a.R % kFirstPix) return cudaErrorInvalidValue;
  dim3 grid((a.R / kFirstPix + 127) / 128, a.R, a.B);
  k_conv_first<C0, T><<<grid, 128, 0, st>>>(a.R, a.cv, a.tiles3,
                                              a.w.w_f32, a.w.gamma, a.w.beta,
                                              static_cast<T*>(a.y), a.y_cs, a.y_co);
  return cudaGetLastError();
}

template <typename T>
cudaError_t first_p(const ConvArgs& a, cudaStream_t st) {
  switch (a.cout) {
    case 8: return first_t<8, T>(a, st);
    case 16: return first_t<16, T>(a, st);
    case 32: return first_t<32, T>(a, st);
    case 64: return first_t<64, T>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_conv_first(const ConvArgs& a, int precision, cudaStream_t st) {
  if (precision == OMNI_FP32) return first_p<float>(a, st);
  return precision == OMNI_FP16 ? first_p<__half>(a, st) : first_p<__nv_bfloat16>(a, st);
}

cudaError_t launch_conv_f32(const ConvArgs& a, cudaStream_t st) {
  if (a.cin % kBK || (a.res_mode == RES_TENSOR && a.cr % kBK)) return cudaErrorInvalidValue;
  long long M = (long long)a.B * a.R * a.R;
  unsigned gx = (unsigned)((M + kBM - 1) / kBM);
  int bn = a.cout >= 64 ? 64 : a.cout;
  if (a.cout % bn) return cudaErrorInvalidValue;
  dim3 grid(gx, a.cout / bn);
  switch (bn) {
    case 64: k_conv_f32<64><<<grid, kThreads, 0, st>>>(a); break;
    case 32: k_conv_f32<32><<<grid, kThreads, 0, st>>>(a); break;
    case 16: k_conv_f32<16><<<grid, kThreads, 0, st>>>(a); break;
    case 8: k_conv_f32<8><<<grid, kThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_maxpool(int precision, int B, int R, int C, const void* x, int x_cs, int x_co,
                           void* y, int y_cs, int y_co, cudaStream_t st) {
  const int n = (R / 2) * (C / 8);
  dim3 grid((n + 127) / 128, R / 2, B);
  if (precision == OMNI_FP32)
    k_maxpool<float><<<grid, 128, 0, st>>>(R, C, (const float*)x, x_cs, x_co, (float*)y, y_cs, y_co);
  else if (precision == OMNI_FP16)
    k_maxpool<__half><<<grid, 128, 0, st>>>(R, C, (const __half*)x, x_cs, x_co, (__half*)y, y_cs, y_co);
  else
    k_maxpool<__nv_bfloat16><<<grid, 128, 0, st>>>(R, C, (const __nv_bfloat16*)x, x_cs, x_co,
                                                   (__nv_bfloat16*)y, y_cs, y_co);
  return cudaGetLastError();
}

cudaError_t launch_upsample(int precision, int B, int R, int C, const void* x, int x_cs,
                            int x_co, void* y, int y_cs, int y_co, cudaStream_t st) {
  if (R % 2 || C % 8) return cudaErrorInvalidValue;
  const int Ri = R / 2;
  const int n = ((Ri + 1 + kUpSeg - 1) / kUpSeg) * (C / 8);
  dim3 grid((n + 127) / 128, Ri + 1, B);
  if (precision == OMNI_FP32)
    k_upsample<float><<<grid, 128, 0, st>>>(Ri, C, (const float*)x, x_cs, x_co, (float*)y, y_cs, y_co);
  else if (precision == OMNI_FP16)
    k_upsample<__half><<<grid, 128, 0, st>>>(Ri, C, (const __half*)x, x_cs, x_co, (__half*)y, y_cs, y_co);
  else
    k_upsample<__nv_bfloat16><<<grid, 128, 0, st>>>(Ri, C, (const __nv_bfloat16*)x, x_cs, x_co,
                                                    (__nv_bfloat16*)y, y_cs, y_co);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- E4M3 experiment
namespace {
// max |x| over n BF16 values, as the bits of a non-negative float (ordered
// like the floats themselves, so atomicMax on the bits is a float max)
__global__ void k_absmax_bf16(const __nv_bfloat16* __restrict__ x, long long n, unsigned* out) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(__bfloat162float(x[i])));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// q = E4M3(x * inv_scale), round to nearest even, saturating at +-448
__global__ void k_quant_e4m3(const __nv_bfloat16* __restrict__ x, long long n, float inv_scale,
                             uint8_t* __restrict__ q) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    q[i] = __nv_cvt_float_to_fp8(__bfloat162float(x[i]) * inv_scale, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float e4m3_amax(const unsigned* amax_bits) {
  const float m = __uint_as_float(*amax_bits);
  return m > 0.f ? m : 448.f;        // an all-zero input keeps scale 1
}

// pixel p's channels c .. c+7 (cin, x_cs, x_co multiples of 8): one 16-byte load
__device__ __forceinline__ void load8_bf16(const __nv_bfloat16* x, long long v, int c8n, int x_cs, int x_co,
                                           float f[8]) {
  const long long pix = v / c8n;
  const int c = (int)(v - pix * c8n) * 8;
  const uint4 u = *reinterpret_cast<const uint4*>(x + pix * x_cs + x_co + c);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 t = __bfloat1622float2(h[k]);
    f[2 * k] = t.x;
    f[2 * k + 1] = t.y;
  }
}

__global__ void k_absmax_strided(const __nv_bfloat16* __restrict__ x, long long npix, int cin, int x_cs,
                                 int x_co, unsigned* out) {
  float m = 0.f;
  const int c8n = cin / 8;
  const long long nv = npix * c8n;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    float f[8];
    load8_bf16(x, v, c8n, x_cs, x_co, f);
#pragma unroll
    for (int k = 0; k < 8; ++k) m = fmaxf(m, fabsf(f[k]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__global__ void k_quant_strided(const __nv_bfloat16* __restrict__ x, long long npix, int cin, int x_cs, int x_co,
                                const unsigned* amax_bits, uint8_t* __restrict__ q) {
  const float inv = 448.f / e4m3_amax(amax_bits);
  const int c8n = cin / 8;
  const long long nv = npix * c8n;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    float f[8];
    load8_bf16(x, v, c8n, x_cs, x_co, f);
    uint32_t w[2] = {0u, 0u};
#pragma unroll
    for (int k = 0; k < 8; ++k)   // channel c + k goes to byte k (little-endian words)
      w[k >> 2] |= (uint32_t)__nv_cvt_float_to_fp8(f[k] * inv, __NV_SATFINITE, __NV_E4M3) << (8 * (k & 3));
    *reinterpret_cast<uint2*>(q + v * 8) = make_uint2(w[0], w[1]);     // q is contiguous [npix][cin]
  }
}

__global__ void k_e4m3_gamma(const float* __restrict__ gamma, const float* __restrict__ s_w, int cout,
                             const unsigned* amax_bits, float* __restrict__ out) {
  const float s_x = e4m3_amax(amax_bits) / 448.f;
  for (int o = threadIdx.x; o < cout; o += blockDim.x) out[o] = gamma[o] * s_w[o] * s_x;
}
}  // namespace

cudaError_t launch_e4m3_activation(const void* x, long long npix, int cin, int x_cs, int x_co,
                                   unsigned* amax_bits, uint8_t* q, const float* gamma, const float* s_w,
                                   int cout, float* gamma_out, cudaStream_t st) {
  if (cin % 8 || x_cs % 8 || x_co % 8 || reinterpret_cast<uintptr_t>(x) % 16 || reinterpret_cast<uintptr_t>(q) % 8)
    return cudaErrorInvalidValue;
  const __nv_bfloat16* xb = static_cast<const __nv_bfloat16*>(x);
  k_absmax_strided<<<1216, 256, 0, st>>>(xb, npix, cin, x_cs, x_co, amax_bits);
  k_quant_strided<<<1216, 256, 0, st>>>(xb, npix, cin, x_cs, x_co, amax_bits, q);
  k_e4m3_gamma<<<1, 512, 0, st>>>(gamma, s_w, cout, amax_bits, gamma_out);
  return cudaGetLastError();
}

cudaError_t launch_absmax_bf16(const void* x, long long n, unsigned* out_bits, cudaStream_t st) {
  k_absmax_bf16<<<1024, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(x), n, out_bits);
  return cudaGetLastError();
}

cudaError_t launch_quant_e4m3(const void* x, long long n, float inv_scale, uint8_t* q, cudaStream_t st) {
  k_quant_e4m3<<<1024, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(x), n, inv_scale, q);
  return cudaGetLastError();
}

}  // namespace omni
