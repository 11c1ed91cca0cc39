// BF16 implicit-GEMM 3x3 convolution of the residual U-Net on the tcgen05
// tensor cores (sm_103a), with the folded norm, the 1x1 residual projection
// and the ReLU fused:  y = ReLU(g * conv3x3(x) + b + wp . r).
//
// GEMM view: M = B*R*R output pixels (NHWC order), N = cout, K = 9*cin
// (tap-major, then channel) for the main segment, plus a second K segment of
// cr channels (the projection, centre tap only) accumulated into its own TMEM
// columns.  A tiles (128 pixels x CK channels) are TMA loads of the shifted
// NHWC input box for each tap; the box runs off the image where the 3x3
// window does, and TMA's zero fill supplies the convolution's zero padding.
// B tiles (BN x CK) are TMA loads of the K-major BF16 weights.
//
// Persistent, warp-specialised CTA (320 threads):
//   warp 0      TMA producer (one elected lane), owns the TMEM allocation
//   warp 1      MMA issuer (one lane): tcgen05.mma M=128 x N=BN x K=16,
//               FP32 accumulators in TMEM, double buffered across tiles
//   warps 2..9  epilogue: tcgen05.ld -> norm, residual, ReLU -> BF16 stores;
//               warps w and w+4 share TMEM lane quarter w%4 and split the
//               columns, so each SM sub-partition interleaves two of them
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA
// records kErrTimeout in the caller's status word, drains its own copies and
// MMAs (again bounded), frees TMEM and returns.
// This file is compiled twice: k_conv_tc.cu (OMNI_TC_F16 = 0, BF16 operands)
// and k_conv_tc_f16.cu (OMNI_TC_F16 = 1, FP16 operands).  The two differ only
// in the MMA operand format and the epilogue's rounding of the output.
#include <cuda.h>
#include <cuda_fp16.h>

#include "omni_internal.cuh"

#ifndef OMNI_TC_F16
#error "define OMNI_TC_F16 before including conv_tc_impl.cuh"
#endif

namespace omni {
namespace {

constexpr bool kF16 = OMNI_TC_F16 != 0;

// two FP32 values rounded to the operand type, packed as one 32-bit word
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (kF16) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

constexpr int kBM = 128;
constexpr int kEpiWarps = 8;                         // two epilogue warpgroups
constexpr int kThreadsTC = 64 + 32 * kEpiWarps;      // producer warp, MMA warp, epilogue
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait
constexpr int kSmemBudget = 222 * 1024;      // per-tap operand slots (+ barriers, norm arrays, alignment)

struct TCParams {
  int B, R, cin, cout, cr;
  int res_mode;
  int n_tiles_m, n_tiles_n, n_tiles;
  int k_main, k_res;                 // K iterations of the two segments
  const float* gamma;
  const float* beta;
  const float* wp_rgb;               // [3][cout] for RES_RGB
  CanvasTab cv;                      // RES_RGB / first layer: canvas of tile b = cv.ptr[tiles3[3 b]]
  const int32_t* tiles3;
  __nv_bfloat16* y;                  // null: output not stored (fused head)
  int y_cs, y_co;
  unsigned* err;
  __nv_bfloat16* pool;               // fused 2x2 max-pool output (small-N kernels) or null
  int pool_cs;
  const float* theta;                // fused pre-head + dynamic heads (kind 1) or null
  const float* wh;
  const float* bh;
  float* logits;
  int slot0, ncls;
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false if the CTA aborted or the limit expired (then sets abort).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned* err) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (now_ns() - t0 > kWaitNs) {
      *abort_flag = 1;
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
}
// Drain wait used after an abort: bounded, ignores the abort flag.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  while (!mbar_try(bar, parity) && now_ns() - t0 < kWaitNs) {
  }
}

// ---- CTA pairs (cluster of two; the pair's MMAs are cta_group::2, M = 256)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
// arrive on a barrier of the other CTA of the pair.  Default (CTA-scope)
// release: a cluster-scope release would first wait until every global store
// of the thread is visible, which the signals here do not need (TMEM reads are
// complete after tcgen05.wait::ld and ordered by the before_thread_sync fence;
// TMA data is tracked by the barrier it completes on).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cl_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cl_addr) : "memory");
}
// arrive on this CTA's barrier (CL false) or on the same barrier of CTA 0 of the pair
template <bool CL>
__device__ __forceinline__ void mbar_arrive_to(uint32_t bar, bool remote) {
  if (CL && remote) mbar_arrive_cluster(cluster_addr(bar, 0));
  else mbar_arrive(bar);
}
// waits on barriers that the other CTA of a pair arrives on: the plain bounded
// wait (the arrivals' ordering is carried by the barrier itself)
template <bool CL>
__device__ __forceinline__ bool mbar_wait_t(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                            unsigned* err) {
  return mbar_wait(bar, parity, abort_flag, err);
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
// tiled shared -> global store of one box; completion is tracked per thread
// with bulk groups (commit, then wait until at most N groups still read smem)
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2,
                                             int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major, swizzled operand tile whose
// rows are SW bytes long (SW = 64 or 128), 8-row groups SW*8 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, int sw) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)1 << 16;                            // leading offset (unused, K-major swizzled)
  d |= (uint64_t)((sw * 8) >> 4) << 32;              // stride offset: next 8-row group
  d |= (uint64_t)1 << 46;                            // descriptor version for tcgen05
  d |= (uint64_t)(sw == 128 ? 2 : 4) << 61;          // swizzle mode: 128B = 2, 64B = 4
  return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 (or FP16 x FP16) -> FP32,
// both operands K-major, M = 128 (256 for a CTA pair).  Operand format
// field: 0 = FP16, 1 = BF16.
__host__ __device__ constexpr uint32_t idesc_bf16(int n, int m = kBM) {
  return (1u << 4) | ((kF16 ? 0u : 1u) << 7) | ((kF16 ? 0u : 1u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// kind::f8f6f4 with E4M3 x E4M3 -> FP32 (operand format code 0 = E4M3), K-major,
// K = 32 per instruction: the same 32 bytes of each operand row as kind::f16
__host__ __device__ constexpr uint32_t idesc_e4m3(int n, int m = kBM) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// pair forms: one MMA over 256 rows (128 from each CTA of the pair; B's N
// columns split N/2 per CTA at the same shared-memory offset), accumulator
// rows in each CTA's own TMEM; the commit arrives on the barrier at the same
// offset in both CTAs
template <bool PAIR, bool F8 = false>
__device__ __forceinline__ void mma_t(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                      uint32_t accumulate) {
  if constexpr (F8) {
    if constexpr (PAIR)
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
          "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
          "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
          : "memory");
    return;
  }
  if (!PAIR) {
    mma_bf16(tmem_d, adesc, bdesc, idesc, accumulate);
    return;
  }
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
template <bool PAIR>
__device__ __forceinline__ void mma_commit_t(uint32_t bar) {
  if (!PAIR) {
    mma_commit(bar);
    return;
  }
  const uint16_t both = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          bar),
      "h"(both)
      : "memory");
}
template <bool PAIR>
__device__ __forceinline__ void tmem_alloc_t(uint32_t slot, uint32_t cols) {
  if (PAIR) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  } else {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}
template <bool PAIR>
__device__ __forceinline__ void tmem_dealloc_t(uint32_t base, uint32_t cols) {
  if (PAIR)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
  else
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane; the
// load and its completion wait are one asm statement so no use of the
// registers can be scheduled before the data has arrived.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Two / three / four 16-column loads issued back to back before a single
// completion wait: the TMEM read latency is paid once per group instead of once
// per load (the epilogues are otherwise bound by those serial waits).
__device__ __forceinline__ void tmem_ld16x2(uint32_t t0, uint32_t t1, float a[16], float b[16]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(t0), "r"(t1)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    a[i] = __uint_as_float(r[i]);
    b[i] = __uint_as_float(r[16 + i]);
  }
}
__device__ __forceinline__ void tmem_ld16x3(uint32_t t0, uint32_t t1, uint32_t t2, float a[16], float b[16],
                                            float c[16]) {
  uint32_t r[48];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%48];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%49];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%50];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
      : "r"(t0), "r"(t1), "r"(t2)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    a[i] = __uint_as_float(r[i]);
    b[i] = __uint_as_float(r[16 + i]);
    c[i] = __uint_as_float(r[32 + i]);
  }
}
__device__ __forceinline__ void tmem_ld16x4(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, float a[16],
                                            float b[16], float c[16], float d[16]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%64];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%65];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%66];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%67];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(t0), "r"(t1), "r"(t2), "r"(t3)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    a[i] = __uint_as_float(r[i]);
    b[i] = __uint_as_float(r[16 + i]);
    c[i] = __uint_as_float(r[32 + i]);
    d[i] = __uint_as_float(r[48 + i]);
  }
}

// v = 2u/255 - 1 for the epilogues' RGB projection: one FMA with the FP32
// constant 2/255, absolute error below 2^-22 like the rounded division it
// replaces (no division sequence per pixel)
__device__ __forceinline__ float norm_u8(uint8_t u) { return fmaf((float)u, 2.0f / 255.0f, -1.0f); }

// four consecutive per-channel constants from shared memory in one 16-byte
// load (the epilogues' gamma / beta / RGB-projection rows are 16-byte aligned)
__device__ __forceinline__ void lds4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

// Dynamic head of one class on the pre-head features h0 of NP pixels (already
// through their ReLU): logit = W3 ReLU(W2 ReLU(W1 h0 + b1) + b2) + b3, with
// theta laid out as W1 (8x8, out-major), W2 (8x8), W3 (8), b1 (8), b2 (8),
// b3 (1).  theta is a 16-byte aligned shared-memory row read with 16-byte
// loads; every weight loaded serves all NP pixels (a broadcast 16-byte load
// costs as many shared-memory wavefronts as four 4-byte ones, so the loads,
// not the FMAs, bound the fused heads).
constexpr int kThetaPad = 168;   // theta row stride of the fused heads' shared copies: the two
                                 // classes' rows start 8 banks apart, so lanes reading different
                                 // classes in one load do not conflict
template <int NP>
__device__ __forceinline__ void dyn_head_n(const float* th, const float (*h0)[8], float* out) {
  const float4* t4 = reinterpret_cast<const float4*>(th);
  float h1[NP][8], h2[NP][8];
  const float4 b1a = t4[34], b1b = t4[35], b2a = t4[36], b2b = t4[37];
  const float b1[8] = {b1a.x, b1a.y, b1a.z, b1a.w, b1b.x, b1b.y, b1b.z, b1b.w};
  const float b2[8] = {b2a.x, b2a.y, b2a.z, b2a.w, b2b.x, b2b.y, b2b.z, b2b.w};
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const float4 wa = t4[2 * o], wb = t4[2 * o + 1];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float* x = h0[q];
      float s = b1[o];
      s = fmaf(wa.x, x[0], s); s = fmaf(wa.y, x[1], s); s = fmaf(wa.z, x[2], s); s = fmaf(wa.w, x[3], s);
      s = fmaf(wb.x, x[4], s); s = fmaf(wb.y, x[5], s); s = fmaf(wb.z, x[6], s); s = fmaf(wb.w, x[7], s);
      h1[q][o] = fmaxf(s, 0.f);
    }
  }
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const float4 wa = t4[16 + 2 * o], wb = t4[16 + 2 * o + 1];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float* x = h1[q];
      float s = b2[o];
      s = fmaf(wa.x, x[0], s); s = fmaf(wa.y, x[1], s); s = fmaf(wa.z, x[2], s); s = fmaf(wa.w, x[3], s);
      s = fmaf(wb.x, x[4], s); s = fmaf(wb.y, x[5], s); s = fmaf(wb.z, x[6], s); s = fmaf(wb.w, x[7], s);
      h2[q][o] = fmaxf(s, 0.f);
    }
  }
  const float4 wa = t4[32], wb = t4[33];
  const float b3 = th[152];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const float* x = h2[q];
    float s = b3;
    s = fmaf(wa.x, x[0], s); s = fmaf(wa.y, x[1], s); s = fmaf(wa.z, x[2], s); s = fmaf(wa.w, x[3], s);
    s = fmaf(wb.x, x[4], s); s = fmaf(wb.y, x[5], s); s = fmaf(wb.z, x[6], s); s = fmaf(wb.w, x[7], s);
    out[q] = s;
  }
}

// Fused pre-head on lane pairs.  Lanes 2i and 2i+1 hold horizontally adjacent
// pixels; lane half h = lane & 1 accumulates pre-head outputs 4h..4h+3 of its
// own pixel (hs) and of its partner's (hp) from the pre-head weights stored
// channel-major (the 8 outputs of a channel contiguous, 16-byte aligned), so a
// lane reads 4 of each channel's 8 weights.  Every output's sum starts from
// its bias and adds the channels in the order one lane doing all eight would.
__device__ __forceinline__ void prehead_pair(const float* swh_t, int n, float v, int h, float hs[4],
                                             float hp[4]) {
  const float vp = __shfl_xor_sync(0xffffffffu, v, 1);
  const float4 w = *reinterpret_cast<const float4*>(swh_t + 8 * n + 4 * h);
  hs[0] = fmaf(w.x, v, hs[0]); hs[1] = fmaf(w.y, v, hs[1]); hs[2] = fmaf(w.z, v, hs[2]); hs[3] = fmaf(w.w, v, hs[3]);
  hp[0] = fmaf(w.x, vp, hp[0]); hp[1] = fmaf(w.y, vp, hp[1]); hp[2] = fmaf(w.z, vp, hp[2]); hp[3] = fmaf(w.w, vp, hp[3]);
}
// ReLU, then one exchange: both lanes of the pair end with all eight pre-head
// outputs of the even lane's pixel (he) and of the odd lane's (ho)
__device__ __forceinline__ void prehead_pair_finish(int h, float hs[4], float hp[4], float he[8], float ho[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hs[k] = fmaxf(hs[k], 0.f);
    hp[k] = fmaxf(hp[k], 0.f);
    const float rs = __shfl_xor_sync(0xffffffffu, hs[k], 1);   // partner's pixel, partner's half
    const float rp = __shfl_xor_sync(0xffffffffu, hp[k], 1);   // this lane's pixel, partner's half
    he[k] = h ? rs : hs[k];
    he[4 + k] = h ? hp[k] : rp;
    ho[k] = h ? rp : hp[k];
    ho[4 + k] = h ? hs[k] : rs;
  }
}

// Dynamic heads of a lane pair's two pixels (he, ho: see prehead_pair_finish)
// into the batch's logit slots at pixel offsets pe / po of the tile image
// whose class-0 plane starts at lo.  Two classes: lane half h runs class h for
// both pixels (one read of its theta row for two pixels), then the pair swaps
// one value so each lane holds both classes of its own pixel and every store
// instruction writes one class plane at the warp's 32 consecutive-row pixels;
// one class: each lane runs it for its own pixel.  A pixel whose write flag is
// off is not stored.
__device__ __forceinline__ void heads_pair(const float* sth, int ncls, long long RR, float* lo, int h,
                                           const float he[8], const float ho[8], long long pe, long long po,
                                           bool we, bool wo) {
  if (ncls == 2) {
    const float x[2][8] = {{he[0], he[1], he[2], he[3], he[4], he[5], he[6], he[7]},
                           {ho[0], ho[1], ho[2], ho[3], ho[4], ho[5], ho[6], ho[7]}};
    float l[2];
    dyn_head_n<2>(sth + h * kThetaPad, x, l);
    // lane 0 of the pair keeps class 0 of the even pixel and receives its class 1;
    // lane 1 keeps class 1 of the odd pixel and receives its class 0
    const float other = __shfl_xor_sync(0xffffffffu, h ? l[0] : l[1], 1);
    const float own = h ? l[1] : l[0];
    const long long pix = h ? po : pe;
    if (h ? wo : we) {
      lo[pix] = h ? other : own;
      lo[RR + pix] = h ? own : other;
    }
  } else {
    float x[1][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[0][k] = h ? ho[k] : he[k];
    float l[1];
    dyn_head_n<1>(sth, x, l);
    if (h ? wo : we) lo[h ? po : pe] = l[0];
  }
}

// 2x2 max of a pixel's 16 channel values with the pixels of lanes lane^dxl
// (horizontal neighbour) and lane^16 (next tile row), rounded and packed
__device__ __forceinline__ void pool_pack(const float v[16], bool down1, uint32_t out[8]) {
  float m[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float h = down1 ? __shfl_down_sync(0xffffffffu, v[j], 1) : __shfl_xor_sync(0xffffffffu, v[j], 1);
    const float a = fmaxf(v[j], h);
    m[j] = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 16));
  }
#pragma unroll
  for (int j = 0; j < 16; j += 2) out[j / 2] = pack2(m[j], m[j + 1]);
}

// Accumulator ring in TMEM: four buffers where they fit in the 512 columns,
// else two, so the MMA warp can run up to three tiles ahead of the epilogue
// (the per-tile handoff latency, not the MMA or the copies, bounds the small
// layers); allocations are a power of two of at least 32 columns.
constexpr int kMaxTmemBufs = 4;
__host__ __device__ constexpr int tmem_bufs(int buf_cols) { return 4 * buf_cols <= 512 ? 4 : 2; }
__host__ __device__ constexpr int tmem_alloc_cols(int cols) {
  return cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
}

// Slot and phase parity of a pipeline ring with a runtime number of stages,
// advanced without division: the producer and MMA roles run on one thread
// each, where a division per step lengthens the whole pipeline.
struct StageRing {
  int s = 0;
  uint32_t ph = 0;
  bool lapped = false;     // every slot has been used once (waits on `empty` begin)
  __device__ __forceinline__ void next(int n) {
    if (++s == n) {
      s = 0;
      ph ^= 1u;
      lapped = true;
    }
  }
};

// This CTA's tiles t = blockIdx.x + i * gridDim.x of an images x ny x nx tile
// grid, kept as (img, ty, tx) and stepped by a mixed-radix add.
// RGB residual input of one epilogue lane, fetched one tile ahead: the
// canvas bytes stay in registers until the tile that needs them, so their
// latency overlaps the current tile instead of following its TMEM wait.
struct RgbPrefetch {
  int t = -1, img = -1, y0 = 0, x0 = 0;
  const uint8_t* base = nullptr;
  long long cs = 0;
  uint32_t b0 = 0, b1 = 0, b2 = 0;
  __device__ __forceinline__ void fetch(const CanvasTab& cv, const int32_t* tiles3, int tile, int im, int hh,
                                        int ww) {
    if (im != img) {
      img = im;
      const int sl = __ldg(tiles3 + 3 * im);
      y0 = __ldg(tiles3 + 3 * im + 1);
      x0 = __ldg(tiles3 + 3 * im + 2);
      base = cv.ptr[sl];
      cs = cv.stride[sl];
    }
    const uint8_t* px = base + (long long)(y0 + hh) * cs + (long long)(x0 + ww) * 3;
    b0 = __ldg(px);
    b1 = __ldg(px + 1);
    b2 = __ldg(px + 2);
    t = tile;
  }
};

struct TileWalk {
  int t, img, ty, tx, step;
  int s_img, s_ty, s_tx, ny, nx;
  // tiles t0, t0 + step, ... (default: this CTA's tiles)
  __device__ __forceinline__ void init(int ny_, int nx_, int t0 = -1, int step_ = 0) {
    ny = ny_;
    nx = nx_;
    const int per = ny * nx;
    t = t0 < 0 ? (int)blockIdx.x : t0;
    step = step_ > 0 ? step_ : (int)gridDim.x;
    img = t / per;
    ty = (t - img * per) / nx;
    tx = t - img * per - ty * nx;
    s_img = step / per;
    s_ty = (step - s_img * per) / nx;
    s_tx = step - s_img * per - s_ty * nx;
  }
  __device__ __forceinline__ void next() {
    t += step;
    tx += s_tx;
    int c = tx >= nx ? 1 : 0;
    tx -= c * nx;
    ty += s_ty + c;
    c = ty >= ny ? 1 : 0;
    ty -= c * ny;
    img += s_img + c;
  }
};

// PAIR: clusters of two CTAs take adjacent M tiles of one N tile; one thread
// of CTA 0 issues cta_group::2 MMAs (M = 256) and each CTA holds half of the
// B tile's rows, so a K step moves a quarter (N = 128) to a third (N = 256)
// less operand data per SM (the wide layers here are bound by that traffic,
// not by the MMA rate)
// F8: E4M3 operands (1 byte per element, K = 32 per MMA); a chunk of CK = 128
// channels is the same 128-byte row as a 64-channel 16-bit chunk
template <int BN, int CK, bool RES, bool PAIR = false, bool F8 = false>
struct TCCfg {
  static constexpr int kEB = F8 ? 1 : 2;                  // operand bytes per element
  static constexpr int kABytes = kBM * CK * kEB;
  static constexpr int kBRows = PAIR ? BN / 2 : BN;       // B rows (output channels) held here
  static constexpr int kBBytes = kBRows * CK * kEB;
  static constexpr int kKSteps = CK * kEB / 32;           // MMAs per K step (32 bytes of K each)
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kStages0 = (kSmemBudget - 2048) / kStageBytes;
  static constexpr int kStages = kStages0 > 16 ? 16 : kStages0;       // (A, B) slots
  // slots per pipeline stage: one wait and one commit cover kGroup K steps,
  // with at least three stages in flight
  static constexpr int kGroup = kStages / 3 > 1 ? kStages / 3 : 1;
  static constexpr int kRing = kStages / kGroup;
  static constexpr int kBufCols = RES ? 2 * BN : BN;     // TMEM columns per accumulator buffer
  static constexpr int kBufs = tmem_bufs(kBufCols);       // accumulator ring depth
  static constexpr int kTmemCols = tmem_alloc_cols(kBufs * kBufCols);
  static constexpr int kSW = CK * kEB;                    // row bytes = swizzle span
  static constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024 /*barriers*/ + 1024 /*align*/ +
                                  2 * 512 * 4 /*gamma, beta*/;
  static_assert(!F8 || !RES, "E4M3 operands: no projection accumulator");
};

template <int BN, int CK, bool RES, bool PAIR, bool F8 = false>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapA2, const __grid_constant__ CUtensorMap mapB2,
              TCParams p) {
  using Cfg = TCCfg<BN, CK, RES, PAIR, F8>;
  constexpr int ST = Cfg::kStages;     // (A, B) slots
  constexpr int G = Cfg::kGroup;       // slots per stage
  constexpr int RING = Cfg::kRing;     // stages
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + (size_t)ST * Cfg::kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)ST * Cfg::kStageBytes);
  uint64_t* full = bars;                 // [ST]
  uint64_t* empty = bars + ST;           // [ST]
  uint64_t* tfull = bars + 2 * ST;                      // [kMaxTmemBufs]
  uint64_t* tempty = bars + 2 * ST + kMaxTmemBufs;      // [kMaxTmemBufs]
  uint64_t* drain = bars + 2 * ST + 2 * kMaxTmemBufs;   // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * ST + 2 * kMaxTmemBufs + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* sg = reinterpret_cast<float*>(smem + (size_t)ST * Cfg::kStageBytes + 1024);   // gamma[cout]
  float* sb = sg + 512;                                                                // beta[cout]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int crank = PAIR ? (int)cluster_rank() : 0;
  const bool peer = crank != 0;                          // CTA 1 of a pair
  // work items: (M tile, N tile); a pair takes M tiles 2 a and 2 a + 1 of one N tile
  const int t_beg = PAIR ? (int)blockIdx.x >> 1 : (int)blockIdx.x;
  const int t_step = PAIR ? (int)gridDim.x >> 1 : (int)gridDim.x;
  const int t_end = PAIR ? p.n_tiles >> 1 : p.n_tiles;
  auto tile_mn = [&](int t, int& mt, int& nt) {
    const int a = t / p.n_tiles_n;
    nt = t - a * p.n_tiles_n;
    mt = PAIR ? 2 * a + crank : a;
  };
  for (int i = threadIdx.x; i < p.cout; i += blockDim.x) {
    sg[i] = p.gamma[i];
    sb[i] = p.beta[i];
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), PAIR && !peer ? 2 : 1);   // pair: plus CTA 1's forwarded loads
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < Cfg::kBufs; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), kEpiWarps * (PAIR ? 2 : 1));
    }
    mbar_init(smem_u32(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (PAIR) cluster_sync();                // both CTAs' barriers exist before any remote arrive
  if (warp == 0) tmem_alloc_t<PAIR>(smem_u32(tmem_slot), Cfg::kTmemCols);
  tc_fence_before();
  if (PAIR) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int k_total = p.k_main + p.k_res;
  const int RR = p.R * p.R;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------------- producer
      int it = 0;
      StageRing ring;
      bool ok = true;
      const int cpt = p.cin / CK;
      for (int tile = t_beg; tile < t_end && ok; tile += t_step) {
        int mt, nt;
        tile_mn(tile, mt, nt);
        const int m0 = mt * kBM;
        const int img = m0 / RR, rem = m0 % RR;
        const int h0 = rem / p.R, w0 = rem % p.R;
        int cc = 0, tdx = 0, tdy = 0;        // channel chunk and tap of the main segment
        for (int k0 = 0; k0 < k_total; k0 += G, ++it, ring.next(RING)) {
          const int s = ring.s;
          if (ring.lapped && !mbar_wait(smem_u32(&empty[s]), ring.ph ^ 1u, abort_flag, p.err)) {
            ok = false;
            break;
          }
          const int nb = min(G, k_total - k0);
          const uint32_t fb = smem_u32(&full[s]);
          mbar_expect_tx(fb, (uint32_t)(nb * Cfg::kStageBytes));
          for (int j = 0; j < nb; ++j) {
            const int k = k0 + j, slot = s * G + j;
            const uint32_t da = smem_u32(sA + (size_t)slot * Cfg::kABytes);
            const uint32_t db = smem_u32(sB + (size_t)slot * Cfg::kBBytes);
            if (k < p.k_main) {
              const int c0 = cc * CK;
              tma_load_4d(da, &mapA, fb, c0, w0 + tdx - 1, h0 + tdy - 1, img);
              tma_load_2d(db, &mapB, fb, (tdy * 3 + tdx) * p.cin + c0, nt * BN + crank * Cfg::kBRows);
              if (++cc == cpt) {
                cc = 0;
                if (++tdx == 3) {
                  tdx = 0;
                  ++tdy;
                }
              }
            } else {
              const int c0 = (k - p.k_main) * CK;
              tma_load_4d(da, &mapA2, fb, c0, w0, h0, img);
              tma_load_2d(db, &mapB2, fb, c0, nt * BN + crank * Cfg::kBRows);
            }
          }
        }
      }
      // make sure no copy of ours is still landing in shared memory
      const int last = it;
      for (int q = last - 1; q >= 0 && q >= last - RING; --q) mbar_drain(smem_u32(&full[q % RING]), (q / RING) & 1);
    }
  } else if (warp == 1 && peer) {
    if (lane == 0) {
      // ---------------------------------------------------------------- pair: forward CTA 1's loads
      // (same stage order as CTA 0's MMA issuer) to CTA 0's stage barriers
      StageRing ring;
      bool ok = true;
      for (int tile = t_beg; tile < t_end && ok; tile += t_step)
        for (int k0 = 0; k0 < k_total; k0 += G, ring.next(RING)) {
          if (!mbar_wait(smem_u32(&full[ring.s]), ring.ph, abort_flag, p.err)) {
            ok = false;
            break;
          }
          mbar_arrive_cluster(cluster_addr(smem_u32(&full[ring.s]), 0));
        }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuer
      constexpr uint32_t idesc = F8 ? idesc_e4m3(BN, PAIR ? 2 * kBM : kBM) : idesc_bf16(BN, PAIR ? 2 * kBM : kBM);
      const uint64_t a_desc0 = smem_desc(smem_u32(sA), Cfg::kSW);
      const uint64_t b_desc0 = smem_desc(smem_u32(sB), Cfg::kSW);
      int tcount = 0;
      StageRing ring;
      bool ok = true;
      for (int tile = t_beg; tile < t_end && ok; tile += t_step, ++tcount) {
        const int buf = tcount % Cfg::kBufs, use = tcount / Cfg::kBufs;
        if (use >= 1 && !mbar_wait(smem_u32(&tempty[buf]), (use - 1) & 1, abort_flag, p.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t acc0 = tmem_base + (uint32_t)(buf * Cfg::kBufCols);
        const uint32_t acc1 = acc0 + BN;
        for (int k0 = 0; k0 < k_total; k0 += G, ring.next(RING)) {
          const int s = ring.s;
          // TMA-filled stage: the mbarrier's complete_tx orders the copy before the MMAs
          if (!mbar_wait(smem_u32(&full[s]), ring.ph, abort_flag, p.err)) {
            ok = false;
            break;
          }
          const int nb = min(G, k_total - k0);
          for (int j = 0; j < nb; ++j) {
            const int k = k0 + j, slot = s * G + j;
            const uint64_t ad = a_desc0 + (uint64_t)(slot * (Cfg::kABytes >> 4));
            const uint64_t bd = b_desc0 + (uint64_t)(slot * (Cfg::kBBytes >> 4));
            const bool second = RES && k >= p.k_main;
            const uint32_t d = second ? acc1 : acc0;
            const int kfirst = second ? p.k_main : 0;
#pragma unroll
            for (int kk = 0; kk < Cfg::kKSteps; ++kk)
              mma_t<PAIR, F8>(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                              (k > kfirst || kk > 0) ? 1u : 0u);
          }
          mma_commit_t<PAIR>(smem_u32(&empty[s]));
        }
        if (!ok) break;
        mma_commit_t<PAIR>(smem_u32(&tfull[buf]));
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit_t<PAIR>(smem_u32(drain));
      mbar_drain(smem_u32(drain), 0);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int q = warp & 3;                  // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    const int c_beg = ((warp - 2) >> 2) * (BN / 2), c_end = c_beg + BN / 2;
    int tcount = 0;
    for (int tile = t_beg; tile < t_end; tile += t_step, ++tcount) {
      const int buf = tcount % Cfg::kBufs, use = tcount / Cfg::kBufs;
      // every lane waits; the vote keeps the warp converged for tcgen05.ld
      const bool ok = mbar_wait(smem_u32(&tfull[buf]), use & 1, abort_flag, p.err);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      int mt, nt;
      tile_mn(tile, mt, nt);
      const long long m = (long long)mt * kBM + row;
      const int n0 = nt * BN;
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      if (p.res_mode == RES_RGB) {
        const int b = (int)(m / RR);
        const int rem = (int)(m - (long long)b * RR);
        const int sl = p.tiles3[3 * b];
        const uint8_t* px = p.cv.ptr[sl] + (long long)(p.tiles3[3 * b + 1] + rem / p.R) * p.cv.stride[sl] +
                            (long long)(p.tiles3[3 * b + 2] + rem % p.R) * 3;
        v0 = norm_u8(px[0]);
        v1 = norm_u8(px[1]);
        v2 = norm_u8(px[2]);
      }
      __nv_bfloat16* out = p.y + m * p.y_cs + p.y_co + n0;
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * Cfg::kBufCols);
#pragma unroll 1
      for (int c = c_beg; c < c_end; c += 16) {
        float a[16], r[16];
        if constexpr (RES) tmem_ld16x2(tb + c, tb + BN + c, a, r);
        else tmem_ld16(tb + c, a);
        uint32_t packed[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          float o[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int n = n0 + c + j + u;
            float z = fmaf(sg[n], a[j + u], sb[n]);
            if constexpr (RES) z += r[j + u];
            if (p.res_mode == RES_RGB)
              z += fmaf(v0, __ldg(p.wp_rgb + n),
                        fmaf(v1, __ldg(p.wp_rgb + p.cout + n), v2 * __ldg(p.wp_rgb + 2 * p.cout + n)));
            o[u] = fmaxf(z, 0.f);
          }
          packed[j / 2] = pack2(o[0], o[1]);
        }
        uint4* dst = reinterpret_cast<uint4*>(out + c);
        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_to<PAIR>(smem_u32(&tempty[buf]), peer);
    }
  }
  __syncwarp();
  tc_fence_before();
  // pair: neither CTA leaves while the other's MMAs or arrivals may still touch it
  if (PAIR) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc_t<PAIR>(tmem_base, Cfg::kTmemCols);
}

// ------------------------------------------------------------------ small-N variant
// For cout <= 64 the A tile of one tap feeds only a few MMA cycles, so the
// per-tap refetch above starves the tensor pipe.  This variant keeps the whole
// layer's weights resident in shared memory (loaded once per CTA) and tiles the
// output as 8 rows x 16 columns.  Per channel chunk it loads three boxes of
// 10 x 16 input pixels, one per horizontal tap offset dx; the operand of tap
// (dy, dx) is rows 16*dy .. 16*dy+127 of box dx, an offset of whole swizzle
// atoms, so nine taps reuse three loads.
constexpr int kHTH = 8, kHTW = 16;
constexpr int kHBoxPix = (kHTH + 2) * kHTW;   // 160 input pixels per dx box

// MB = 2: a tile is two vertically adjacent 8 x 16 blocks (16 x 16 pixels);
// the boxes are 18 rows high and every synchronisation of the pipeline
// covers twice the MMAs (the per-tile waits dominate at small N).
//
// PAIR: the kernel runs as clusters of two CTAs.  Each CTA loads and stores
// its own tiles (CTA 0 of the pair the even, CTA 1 the odd tiles of the pair's
// sequence) and holds half of the weights' N rows; one thread of CTA 0 issues
// cta_group::2 MMAs of M = 256 that cover the same block of both CTAs' tiles,
// so an instruction does twice the rows for the same issue cost (at N = 32 /
// 64 an MMA's issue cost, not its math, bounds the layer).  CTA 1's idle MMA
// warp forwards its loads' completion to CTA 0's stage barriers; the MMA
// commits arrive on both CTAs' barriers; both epilogues release an
// accumulator buffer on CTA 0's barrier.
template <int BN, int CK, bool RES, int MB, bool PAIR = false>
struct HaloCfg {
  static constexpr int kBoxRows = kHTH * MB + 2;
  static constexpr int kBoxBytes = kBoxRows * kHTW * CK * 2;
  static constexpr int kStageBytes = 3 * kBoxBytes;
  static constexpr int kWRows = PAIR ? BN / 2 : BN;      // weight rows (output channels) held here
  static constexpr int kWTileBytes = kWRows * CK * 2;
  static constexpr int kBlkCols = RES ? 2 * BN : BN;     // one 128-pixel block: conv | projection
  static constexpr int kBufCols = MB * kBlkCols;
  static constexpr int kBufs = tmem_bufs(kBufCols);
  static constexpr int kTmemCols = tmem_alloc_cols(kBufs * kBufCols);
  static constexpr int kSW = CK * 2;
};

struct HaloParams {
  TCParams t;                       // t.k_res = slots of the projection segment (3 chunks each)
  int res_chunks;                   // channel chunks of the projection input
  int stages, n_wtiles, cpt;        // stages of the ring; cpt = channel chunks of the main input
  int tiles_per_img, tiles_w;       // (R/(8 MB))*(R/16), R/16
  int group;                        // slots (one chunk's 3 boxes, or 3 projection chunks) per stage
};

template <int BN, int CK, bool RES, int MB, bool PAIR>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_conv_tc_halo(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapA2, const __grid_constant__ CUtensorMap mapB2,
                   HaloParams hp) {
  using Cfg = HaloCfg<BN, CK, RES, MB, PAIR>;
  const TCParams& p = hp.t;
  const int ST = hp.stages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sW = smem;
  uint8_t* sA = smem + (size_t)hp.n_wtiles * Cfg::kWTileBytes;
  const int G = hp.group;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + (size_t)ST * G * Cfg::kStageBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + ST;
  uint64_t* tfull = bars + 2 * ST;                      // [kMaxTmemBufs]
  uint64_t* tempty = bars + 2 * ST + kMaxTmemBufs;      // [kMaxTmemBufs]
  uint64_t* drain = bars + 2 * ST + 2 * kMaxTmemBufs;
  uint64_t* wbar = bars + 2 * ST + 2 * kMaxTmemBufs + 1;
  float* sg = reinterpret_cast<float*>(bars + 2 * ST + 2 * kMaxTmemBufs + 2);    // gamma[BN]
  float* sb = sg + BN;                                          // beta[BN]
  float* swp = sb + BN;                                         // wp_rgb[3][BN]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(swp + 3 * BN);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* swh = reinterpret_cast<float*>(tmem_slot + 4);             // fused head: wh as [BN][8]
  float* sbh = swh + kHeadCh * BN;                                  // bh[8]
  float* sthe = sbh + kHeadCh;                                      // theta rows per epilogue warp

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool fuse_head = p.theta != nullptr;
  const bool peer = PAIR && cluster_rank() != 0;          // CTA 1 of a pair
  for (int i = threadIdx.x; i < BN; i += blockDim.x) {
    sg[i] = p.gamma[i];
    sb[i] = p.beta[i];
    if (p.res_mode == RES_RGB) {
      swp[i] = p.wp_rgb[i];
      swp[BN + i] = p.wp_rgb[p.cout + i];
      swp[2 * BN + i] = p.wp_rgb[2 * p.cout + i];
    }
  }
  if (fuse_head) {
    for (int i = threadIdx.x; i < kHeadCh * BN; i += blockDim.x) swh[(i % BN) * kHeadCh + i / BN] = p.wh[i];
    if (threadIdx.x < kHeadCh) sbh[threadIdx.x] = p.bh[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    // pair, CTA 0: the stage and weight barriers also wait for CTA 1's
    // forwarded completion, the accumulator buffers for both epilogues
    const uint32_t fwd = PAIR && !peer ? 2 : 1;
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), fwd);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < Cfg::kBufs; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      // one block: with the fused head each warpgroup owns the buffers of one parity
      mbar_init(smem_u32(&tempty[b]), (MB == 1 && fuse_head ? kEpiWarps / 2 : kEpiWarps) * (PAIR ? 2 : 1));
    }
    mbar_init(smem_u32(drain), 1);
    mbar_init(smem_u32(wbar), fwd);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (PAIR) cluster_sync();                // both CTAs' barriers exist before any remote arrive
  if (warp == 0) tmem_alloc_t<PAIR>(smem_u32(tmem_slot), Cfg::kTmemCols);
  tc_fence_before();
  if (PAIR) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int k_total = p.k_main + p.k_res;
  const int RR = p.R * p.R;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------------- producer
      const uint32_t wb = smem_u32(wbar);
      mbar_expect_tx(wb, (uint32_t)(hp.n_wtiles * Cfg::kWTileBytes));
      for (int t = 0; t < 9 * hp.cpt; ++t) {
        const int tap = t / hp.cpt, c = t % hp.cpt;
        tma_load_2d(smem_u32(sW + (size_t)t * Cfg::kWTileBytes), &mapB, wb, tap * p.cin + c * CK,
                    peer ? Cfg::kWRows : 0);
      }
      for (int r = 0; r < hp.res_chunks; ++r)
        tma_load_2d(smem_u32(sW + (size_t)(9 * hp.cpt + r) * Cfg::kWTileBytes), &mapB2, wb, r * CK,
                    peer ? Cfg::kWRows : 0);
      int it = 0;
      StageRing ring;
      TileWalk tw;
      tw.init(hp.tiles_per_img / hp.tiles_w, hp.tiles_w);
      bool ok = true;
      for (; tw.t < p.n_tiles && ok; tw.next()) {
        const int img = tw.img;
        const int h0 = tw.ty * (kHTH * MB), w0 = tw.tx * kHTW;
        for (int k0 = 0; k0 < k_total; k0 += G, ++it, ring.next(ST)) {
          const int s = ring.s;
          if (ring.lapped && !mbar_wait_t<PAIR>(smem_u32(&empty[s]), ring.ph ^ 1u, abort_flag, p.err)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full[s]);
          const int nsl = min(G, k_total - k0);
          uint32_t bytes = 0;
          for (int j = 0; j < nsl; ++j) {
            const int k = k0 + j;
            bytes += k < p.k_main ? (uint32_t)Cfg::kStageBytes
                                  : (uint32_t)(min(3, hp.res_chunks - (k - p.k_main) * 3) * MB * kBM * CK * 2);
          }
          mbar_expect_tx(fb, bytes);
          for (int j = 0; j < nsl; ++j) {
            const int k = k0 + j;
            uint8_t* st = sA + (size_t)(s * G + j) * Cfg::kStageBytes;
            if (k < p.k_main) {
              const int c0 = k * CK;
              for (int dx = 0; dx < 3; ++dx)
                tma_load_4d(smem_u32(st + dx * Cfg::kBoxBytes), &mapA, fb, c0, w0 + dx - 1, h0 - 1, img);
            } else {
              // up to three projection chunks per slot, one per box
              const int c0 = (k - p.k_main) * 3, nbx = min(3, hp.res_chunks - c0);
              for (int b = 0; b < nbx; ++b)
                tma_load_4d(smem_u32(st + b * Cfg::kBoxBytes), &mapA2, fb, (c0 + b) * CK, w0, h0, img);
            }
          }
        }
      }
      const int last = it;
      for (int q = last - 1; q >= 0 && q >= last - ST; --q) mbar_drain(smem_u32(&full[q % ST]), (q / ST) & 1);
      mbar_drain(wb, 0);
    }
  } else if (warp == 1 && peer) {
    if (lane == 0) {
      // ---------------------------------------------------------------- pair: forward CTA 1's loads
      // (same stage order as CTA 0's MMA issuer) to CTA 0's barriers
      bool ok = mbar_wait(smem_u32(wbar), 0, abort_flag, p.err);
      if (ok) mbar_arrive_cluster(cluster_addr(smem_u32(wbar), 0));
      StageRing ring;
      for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x)
        for (int k0 = 0; k0 < k_total; k0 += G, ring.next(ST)) {
          if (!mbar_wait(smem_u32(&full[ring.s]), ring.ph, abort_flag, p.err)) {
            ok = false;
            break;
          }
          mbar_arrive_cluster(cluster_addr(smem_u32(&full[ring.s]), 0));
        }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BN, PAIR ? 2 * kBM : kBM);
      const uint64_t a_desc0 = smem_desc(smem_u32(sA), Cfg::kSW);
      const uint64_t b_desc0 = smem_desc(smem_u32(sW), Cfg::kSW);
      const uint64_t b_tap_step = (uint64_t)(hp.cpt * (Cfg::kWTileBytes >> 4));
      bool ok = mbar_wait_t<PAIR>(smem_u32(wbar), 0, abort_flag, p.err);
      int tcount = 0;
      StageRing ring;
      for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x, ++tcount) {
        const int buf = tcount % Cfg::kBufs, use = tcount / Cfg::kBufs;
        if (use >= 1 && !mbar_wait_t<PAIR>(smem_u32(&tempty[buf]), (use - 1) & 1, abort_flag, p.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t acc0 = tmem_base + (uint32_t)(buf * Cfg::kBufCols);
        const uint32_t acc1 = acc0 + BN;
        for (int k0 = 0; k0 < k_total; k0 += G, ring.next(ST)) {
          const int s = ring.s;
          // TMA-filled stage: the mbarrier's complete_tx orders the copy before the MMAs
          if (!mbar_wait_t<PAIR>(smem_u32(&full[s]), ring.ph, abort_flag, p.err)) {
            ok = false;
            break;
          }
          const int nsl = min(G, k_total - k0);
          for (int j = 0; j < nsl; ++j) {
            const int k = k0 + j;
            // descriptor start addresses advance in 16-byte units: add (bytes >> 4)
            const uint64_t ad = a_desc0 + (uint64_t)(((s * G + j) * Cfg::kStageBytes) >> 4);
            if (k < p.k_main) {
              const uint64_t bd = b_desc0 + (uint64_t)(k * (Cfg::kWTileBytes >> 4));
              const uint32_t acc_first = k > 0 ? 1u : 0u;
#pragma unroll
              for (int blk = 0; blk < MB; ++blk) {
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                  // tap (dy, dx): box dx, rows dy + 8 blk .. (whole swizzle atoms)
                  const uint64_t at = ad + (uint64_t)(((tap % 3) * Cfg::kBoxBytes +
                                                       (tap / 3 + kHTH * blk) * kHTW * CK * 2) >> 4);
                  const uint64_t bt = bd + (uint64_t)tap * b_tap_step;
#pragma unroll
                  for (int kk = 0; kk < CK / 16; ++kk)
                    mma_t<PAIR>(acc0 + (uint32_t)(blk * Cfg::kBlkCols), at + (uint64_t)(kk * 2),
                                bt + (uint64_t)(kk * 2), idesc, (tap > 0 || kk > 0) ? 1u : acc_first);
                }
              }
            } else if (RES) {
              const int c0 = (k - p.k_main) * 3, nbx = min(3, hp.res_chunks - c0);
              for (int b = 0; b < nbx; ++b) {
                const uint64_t bd = b_desc0 + (uint64_t)((9 * hp.cpt + c0 + b) * (Cfg::kWTileBytes >> 4));
#pragma unroll
                for (int blk = 0; blk < MB; ++blk) {
                  const uint64_t ab =
                      ad + (uint64_t)((b * Cfg::kBoxBytes + kHTH * blk * kHTW * CK * 2) >> 4);
#pragma unroll
                  for (int kk = 0; kk < CK / 16; ++kk)
                    mma_t<PAIR>(acc1 + (uint32_t)(blk * Cfg::kBlkCols), ab + (uint64_t)(kk * 2),
                                bd + (uint64_t)(kk * 2), idesc, (c0 + b > 0 || kk > 0) ? 1u : 0u);
                }
              }
            }
          }
          mma_commit_t<PAIR>(smem_u32(&empty[s]));
        }
        if (!ok) break;
        mma_commit_t<PAIR>(smem_u32(&tfull[buf]));
      }
      mma_commit_t<PAIR>(smem_u32(drain));
      mbar_drain(smem_u32(drain), 0);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    // Default: warps w and w+4 share TMEM lane quarter w%4 and split the
    // columns.  Fused head: each warpgroup owns the TMEM buffers of one parity
    // (alternate tiles) and reads every column, so a thread holds its pixel.
    // MB = 2: warpgroup g takes block g of every tile, all columns.
    const int q = warp & 3, grp = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const bool split = MB == 1 && !fuse_head;
    const int blk = MB == 2 ? grp : 0;
    const int c_beg = split ? grp * (BN / 2) : 0, c_end = split ? c_beg + BN / 2 : BN;
    const int Rh = p.R >> 1;
    float* sth = sthe + (warp - 2) * (2 * kThetaPad);
    int th_img = -1;
    int tcount = 0;
    const bool rgb = p.res_mode == RES_RGB;
    RgbPrefetch pf;
    TileWalk tw;
    tw.init(hp.tiles_per_img / hp.tiles_w, hp.tiles_w);
    for (; tw.t < p.n_tiles; tw.next(), ++tcount) {
      const int buf = tcount % Cfg::kBufs, use = tcount / Cfg::kBufs;
      if (MB == 1 && fuse_head && (buf & 1) != grp) continue;
      uint32_t u0 = 0, u1 = 0, u2 = 0;
      if (rgb) {
        if (pf.t != tw.t)
          pf.fetch(p.cv, p.tiles3, tw.t, tw.img,
                   tw.ty * (kHTH * MB) + blk * kHTH + row / kHTW, tw.tx * kHTW + row % kHTW);
        u0 = pf.b0; u1 = pf.b1; u2 = pf.b2;
        TileWalk nx = tw;
        nx.next();
        if (nx.t < p.n_tiles)
          pf.fetch(p.cv, p.tiles3, nx.t, nx.img,
                   nx.ty * (kHTH * MB) + blk * kHTH + row / kHTW, nx.tx * kHTW + row % kHTW);
      }
      const bool ok = mbar_wait_t<PAIR>(smem_u32(&tfull[buf]), use & 1, abort_flag, p.err);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int img = tw.img;
      const int hh = tw.ty * (kHTH * MB) + blk * kHTH + row / kHTW;
      const int ww = tw.tx * kHTW + row % kHTW;
      const long long m = (long long)img * RR + (long long)hh * p.R + ww;
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      if (rgb) {
        v0 = norm_u8((uint8_t)u0);
        v1 = norm_u8((uint8_t)u1);
        v2 = norm_u8((uint8_t)u2);
      }
      // fused head: this lane's half of the pre-head outputs for its pixel and its partner's
      const int hf = lane & 1;
      float hs[4], hp[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) hs[k] = hp[k] = fuse_head ? sbh[4 * hf + k] : 0.f;
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) +
                          (uint32_t)(buf * Cfg::kBufCols + blk * Cfg::kBlkCols);
#pragma unroll 1
      for (int c = c_beg; c < c_end; c += 16) {
        float a[16], r[16], o16[16];
        if constexpr (RES) tmem_ld16x2(tb + c, tb + BN + c, a, r);
        else tmem_ld16(tb + c, a);
#pragma unroll
        for (int j4 = 0; j4 < 16; j4 += 4) {
          float g4[4], b4[4], w0[4] = {0.f, 0.f, 0.f, 0.f}, w1[4] = {0.f, 0.f, 0.f, 0.f},
                                 w2[4] = {0.f, 0.f, 0.f, 0.f};
          lds4(sg + c + j4, g4);
          lds4(sb + c + j4, b4);
          if (rgb) {
            lds4(swp + c + j4, w0);
            lds4(swp + BN + c + j4, w1);
            lds4(swp + 2 * BN + c + j4, w2);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j4 + u;
            float z = fmaf(g4[u], a[j], b4[u]);
            if constexpr (RES) z += r[j];
            if (rgb) z += fmaf(v0, w0[u], fmaf(v1, w1[u], v2 * w2[u]));
            o16[j] = fmaxf(z, 0.f);
          }
        }
        if (p.y) {
          uint32_t packed[8];
#pragma unroll
          for (int j = 0; j < 16; j += 2) packed[j / 2] = pack2(o16[j], o16[j + 1]);
          uint4* dst = reinterpret_cast<uint4*>(p.y + m * p.y_cs + p.y_co + c);
          dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
        if (p.pool) {
          // lanes 0-15 / 16-31 hold tile rows 2k / 2k+1 (even row and column origins)
          uint32_t pk[8];
          pool_pack(o16, false, pk);
          if ((lane & 17) == 0) {
            uint4* dst = reinterpret_cast<uint4*>(
                p.pool + (((long long)img * Rh + (hh >> 1)) * Rh + (ww >> 1)) * p.pool_cs + c);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          }
        }
        if (fuse_head) {
#pragma unroll
          for (int j = 0; j < 16; ++j) prehead_pair(swh, c + j, o16[j], hf, hs, hp);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_to<PAIR>(smem_u32(&tempty[buf]), peer);
      if (fuse_head) {
        // the TMEM buffer is released; the heads run on registers and shared memory
        float he[8], ho[8];
        prehead_pair_finish(hf, hs, hp, he, ho);
        if (img != th_img) {
          __syncwarp();
          const float* src = p.theta + (long long)img * p.ncls * kHeadParams;
          for (int i = lane; i < p.ncls * kHeadParams; i += 32) sth[(i / kHeadParams) * kThetaPad + i % kHeadParams] = src[i];
          __syncwarp();
          th_img = img;
        }
        // the pair's pixels are columns ww and ww ^ 1 of tile row hh
        const long long pix = (long long)hh * p.R + ww, pix_p = (long long)hh * p.R + (ww ^ 1);
        heads_pair(sth, p.ncls, RR, p.logits + (long long)(p.slot0 + img) * p.ncls * RR, hf, he, ho,
                   hf ? pix_p : pix, hf ? pix : pix_p, true, true);
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  // pair: neither CTA leaves while the other's MMAs or arrivals may still touch it
  if (PAIR) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc_t<PAIR>(tmem_base, Cfg::kTmemCols);
}

// ------------------------------------------------------------------ dx-in-N variant
// Pixels stay on M (128 = 8 rows x 16 columns), but the three horizontal taps
// move to N: B stacks the weights of dx = 0, 1, 2 (N = 3 * cout), so one MMA of
// tap row dy computes D[p][(dx, co)] for the unshifted input rows.  A is a
// single box of 10 x 16 input pixels per channel chunk, whose three dy views
// are 16-row (whole swizzle atom) offsets.  The output at column c of a tile
// row is D0[c-1] + D1[c] + D2[c+1]: a horizontal pixel shift is a neighbouring
// TMEM lane inside a 16-lane row group, so the epilogue sums the three dx
// blocks with +-1 lane warp shuffles.  Tiles advance by 14 columns and keep
// one halo column on each side (lanes 0 and 15 of each row group write nothing).
constexpr int kXTW = 14;                       // valid output columns per tile row

// MB = 2: two vertically adjacent 8-row blocks per tile (16 x 14 outputs),
// 18-row boxes, one pipeline synchronisation per two blocks.
template <int CO, int CK, bool RES, int MB>
struct DxnCfg {
  static constexpr int kN = 3 * CO;                        // MMA N (dx blocks)
  static constexpr int kBoxRows = kHTH * MB + 2;
  static constexpr int kBoxBytes = kBoxRows * kHTW * CK * 2;
  static constexpr int kStageBytes = kBoxBytes;            // one box slot (a stage holds cps slots)
  static constexpr int kWTileBytes = kN * CK * 2;          // 3 dx slices of cout x CK
  static constexpr int kRTileBytes = CO * CK * 2;          // projection weights
  static constexpr int kBlkCols = RES ? kN + CO : kN;      // one 128-lane block: dx blocks | projection
  static constexpr int kBufCols = MB * kBlkCols;
  static constexpr int kBufs = tmem_bufs(kBufCols);
  static constexpr int kTmemCols = tmem_alloc_cols(kBufs * kBufCols);
  static constexpr int kSW = CK * 2;
};

struct DxnParams {
  TCParams t;
  int res_chunks, stages, cpt;
  int tiles_per_img, tiles_w;      // (R/8) * ceil(R/14), ceil(R/14)
  int wbytes;                      // resident weight bytes (main + projection)
  int cps;                         // slots per pipeline stage; a tile has cpt + res_chunks slots
};

template <int CO, int CK, bool RES, int MB>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_conv_tc_dxn(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ CUtensorMap mapA2, const __grid_constant__ CUtensorMap mapB2,
                  DxnParams hp) {
  using Cfg = DxnCfg<CO, CK, RES, MB>;
  const TCParams& p = hp.t;
  const int ST = hp.stages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sW = smem;                                              // [3 dy][cpt][3 cout x CK]
  uint8_t* sR = sW + (size_t)9 * hp.cpt * Cfg::kRTileBytes;        // [res_chunks][cout x CK]
  uint8_t* sA = smem + hp.wbytes;
  const int stage_bytes = hp.cps * Cfg::kStageBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + (size_t)ST * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + ST;
  uint64_t* tfull = bars + 2 * ST;                      // [kMaxTmemBufs]
  uint64_t* tempty = bars + 2 * ST + kMaxTmemBufs;      // [kMaxTmemBufs]
  uint64_t* drain = bars + 2 * ST + 2 * kMaxTmemBufs;
  uint64_t* wbar = bars + 2 * ST + 2 * kMaxTmemBufs + 1;
  float* sg = reinterpret_cast<float*>(bars + 2 * ST + 2 * kMaxTmemBufs + 2);
  float* sb = sg + CO;
  float* swp = sb + CO;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(swp + 3 * CO);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* swh = reinterpret_cast<float*>(tmem_slot + 4);             // fused head: wh as [CO][8]
  float* sbh = swh + kHeadCh * CO;                                  // bh[8]
  float* sthe = sbh + kHeadCh;                                      // theta rows per epilogue warp

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool fuse_head = p.theta != nullptr;
  for (int i = threadIdx.x; i < CO; i += blockDim.x) {
    sg[i] = p.gamma[i];
    sb[i] = p.beta[i];
    if (p.res_mode == RES_RGB) {
      swp[i] = p.wp_rgb[i];
      swp[CO + i] = p.wp_rgb[p.cout + i];
      swp[2 * CO + i] = p.wp_rgb[2 * p.cout + i];
    }
  }
  if (fuse_head) {
    for (int i = threadIdx.x; i < kHeadCh * CO; i += blockDim.x) swh[(i % CO) * kHeadCh + i / CO] = p.wh[i];
    if (threadIdx.x < kHeadCh) sbh[threadIdx.x] = p.bh[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < Cfg::kBufs; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      // one block with the fused head: each warpgroup owns the buffers of one parity
      mbar_init(smem_u32(&tempty[b]), MB == 1 && fuse_head ? kEpiWarps / 2 : kEpiWarps);
    }
    mbar_init(smem_u32(drain), 1);
    mbar_init(smem_u32(wbar), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(Cfg::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int k_total = p.k_main + p.k_res;
  const int RR = p.R * p.R;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------------- producer
      const uint32_t wb = smem_u32(wbar);
      mbar_expect_tx(wb, (uint32_t)hp.wbytes);
      for (int dy = 0; dy < 3; ++dy)
        for (int c = 0; c < hp.cpt; ++c)
          for (int dx = 0; dx < 3; ++dx)
            tma_load_2d(smem_u32(sW + (size_t)(dy * hp.cpt + c) * Cfg::kWTileBytes + dx * Cfg::kRTileBytes),
                        &mapB, wb, (dy * 3 + dx) * p.cin + c * CK, 0);
      for (int r = 0; r < hp.res_chunks; ++r)
        tma_load_2d(smem_u32(sR + (size_t)r * Cfg::kRTileBytes), &mapB2, wb, r * CK, 0);
      int it = 0;
      StageRing ring;
      TileWalk tw;
      tw.init(hp.tiles_per_img / hp.tiles_w, hp.tiles_w);
      bool ok = true;
      for (; tw.t < p.n_tiles && ok; tw.next()) {
        const int img = tw.img;
        const int h0 = tw.ty * (kHTH * MB), w0 = tw.tx * kXTW;
        // slots of a tile: cpt main chunks, then res_chunks projection chunks;
        // a stage carries cps consecutive slots
        for (int k0 = 0; k0 < k_total; k0 += hp.cps, ++it, ring.next(ST)) {
          const int s = ring.s;
          if (ring.lapped && !mbar_wait(smem_u32(&empty[s]), ring.ph ^ 1u, abort_flag, p.err)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full[s]);
          uint8_t* st = sA + (size_t)s * stage_bytes;
          const int nb = min(hp.cps, k_total - k0);
          uint32_t bytes = 0;
          for (int j = 0; j < nb; ++j)
            bytes += k0 + j < hp.cpt ? (uint32_t)Cfg::kBoxBytes : (uint32_t)(MB * kBM * CK * 2);
          mbar_expect_tx(fb, bytes);
          for (int j = 0; j < nb; ++j) {
            const int k = k0 + j;
            if (k < hp.cpt)
              tma_load_4d(smem_u32(st + j * Cfg::kBoxBytes), &mapA, fb, k * CK, w0 - 1, h0 - 1, img);
            else
              tma_load_4d(smem_u32(st + j * Cfg::kBoxBytes), &mapA2, fb, (k - hp.cpt) * CK, w0 - 1, h0, img);
          }
        }
      }
      const int last = it;
      for (int q = last - 1; q >= 0 && q >= last - ST; --q) mbar_drain(smem_u32(&full[q % ST]), (q / ST) & 1);
      mbar_drain(wb, 0);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuer
      constexpr uint32_t idesc_n = idesc_bf16(Cfg::kN);
      constexpr uint32_t idesc_r = idesc_bf16(CO);
      const uint64_t a_desc0 = smem_desc(smem_u32(sA), Cfg::kSW);
      const uint64_t w_desc0 = smem_desc(smem_u32(sW), Cfg::kSW);
      const uint64_t r_desc0 = smem_desc(smem_u32(sR), Cfg::kSW);
      const uint64_t dy_step = (uint64_t)(hp.cpt * (Cfg::kWTileBytes >> 4));
      bool ok = mbar_wait(smem_u32(wbar), 0, abort_flag, p.err);
      int tcount = 0;
      StageRing ring;
      for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x, ++tcount) {
        const int buf = tcount % Cfg::kBufs, use = tcount / Cfg::kBufs;
        if (use >= 1 && !mbar_wait(smem_u32(&tempty[buf]), (use - 1) & 1, abort_flag, p.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t acc0 = tmem_base + (uint32_t)(buf * Cfg::kBufCols);
        const uint32_t acc1 = acc0 + Cfg::kN;
        for (int k0 = 0; k0 < k_total; k0 += hp.cps, ring.next(ST)) {
          const int s = ring.s;
          // TMA-filled stage: the mbarrier's complete_tx orders the copy before the MMAs
          if (!mbar_wait(smem_u32(&full[s]), ring.ph, abort_flag, p.err)) {
            ok = false;
            break;
          }
          const uint64_t ad = a_desc0 + (uint64_t)((s * stage_bytes) >> 4);
          const int nb = min(hp.cps, k_total - k0);
          // the stage's main slots, then its projection slots: no branch between MMAs
          const int nmain = RES ? max(0, min(nb, hp.cpt - k0)) : nb;
          for (int j = 0; j < nmain; ++j) {
            const int c = k0 + j;
            const uint64_t aj = ad + (uint64_t)((j * Cfg::kBoxBytes) >> 4);
            const uint64_t bk = w_desc0 + (uint64_t)(c * (Cfg::kWTileBytes >> 4));
#pragma unroll
            for (int blk = 0; blk < MB; ++blk) {
#pragma unroll
              for (int dy = 0; dy < 3; ++dy) {
                const uint64_t at = aj + (uint64_t)(((dy + kHTH * blk) * kHTW * CK * 2) >> 4);
                const uint64_t bt = bk + (uint64_t)dy * dy_step;
#pragma unroll
                for (int kk = 0; kk < CK / 16; ++kk)
                  mma_bf16(acc0 + (uint32_t)(blk * Cfg::kBlkCols), at + (uint64_t)(kk * 2),
                           bt + (uint64_t)(kk * 2), idesc_n, (c > 0 || dy > 0 || kk > 0) ? 1u : 0u);
              }
            }
          }
          if constexpr (RES) {
            for (int j = nmain; j < nb; ++j) {
              const int r = k0 + j - hp.cpt;
              const uint64_t bd = r_desc0 + (uint64_t)(r * (Cfg::kRTileBytes >> 4));
#pragma unroll
              for (int blk = 0; blk < MB; ++blk) {
                const uint64_t aj =
                    ad + (uint64_t)((j * Cfg::kBoxBytes + kHTH * blk * kHTW * CK * 2) >> 4);
#pragma unroll
                for (int kk = 0; kk < CK / 16; ++kk)
                  mma_bf16(acc1 + (uint32_t)(blk * Cfg::kBlkCols), aj + (uint64_t)(kk * 2),
                           bd + (uint64_t)(kk * 2), idesc_r, (r > 0 || kk > 0) ? 1u : 0u);
              }
            }
          }
          mma_commit(smem_u32(&empty[s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&tfull[buf]));
      }
      mma_commit(smem_u32(drain));
      mbar_drain(smem_u32(drain), 0);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    // MB = 1: warps w and w+4 share lane quarter w%4 and split the output
    // channels, or, with the fused head (a thread needs all channels of its
    // pixel), warpgroup g takes the TMEM buffers of parity g (alternate
    // tiles) whole; MB = 2: warpgroup g takes block g, all channels
    const int q = warp & 3, grp = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const int col = row % kHTW;                        // column inside the 16-lane row group
    const int blk = MB == 2 ? grp : 0;
    const bool split = MB == 1 && !fuse_head;
    const int co_beg = split ? grp * (CO / 2) : 0, co_end = split ? co_beg + CO / 2 : CO;
    float* sth = sthe + (warp - 2) * (2 * kThetaPad);
    int th_img = -1;
    int tcount = 0;
    const bool rgb = p.res_mode == RES_RGB;
    RgbPrefetch pf;
    TileWalk tw;
    tw.init(hp.tiles_per_img / hp.tiles_w, hp.tiles_w);
    for (; tw.t < p.n_tiles; tw.next(), ++tcount) {
      const int buf = tcount % Cfg::kBufs, use = tcount / Cfg::kBufs;
      if (MB == 1 && fuse_head && (buf & 1) != grp) continue;
      uint32_t u0 = 0, u1 = 0, u2 = 0;
      if (rgb) {
        // lanes without an output column (halo lanes, columns past R) fetch nothing
        const int wc = tw.tx * kXTW + col - 1;
        if (pf.t != tw.t && col >= 1 && col <= kXTW && wc < p.R)
          pf.fetch(p.cv, p.tiles3, tw.t, tw.img,
                   tw.ty * (kHTH * MB) + blk * kHTH + row / kHTW, wc);
        u0 = pf.b0; u1 = pf.b1; u2 = pf.b2;
        TileWalk nx = tw;
        nx.next();
        const int wn = nx.tx * kXTW + col - 1;
        if (nx.t < p.n_tiles && col >= 1 && col <= kXTW && wn < p.R)
          pf.fetch(p.cv, p.tiles3, nx.t, nx.img,
                   nx.ty * (kHTH * MB) + blk * kHTH + row / kHTW, wn);
      }
      const bool ok = mbar_wait(smem_u32(&tfull[buf]), use & 1, abort_flag, p.err);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int img = tw.img;
      const int hh = tw.ty * (kHTH * MB) + blk * kHTH + row / kHTW;
      const int ww = tw.tx * kXTW + col - 1;                        // this lane's pixel column
      const bool writes = col >= 1 && col <= kXTW && ww < p.R;
      const long long m = (long long)img * RR + (long long)hh * p.R + (ww < 0 ? 0 : ww);
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      if (rgb && writes) {
        v0 = norm_u8((uint8_t)u0);
        v1 = norm_u8((uint8_t)u1);
        v2 = norm_u8((uint8_t)u2);
      }
      __nv_bfloat16* out = p.y + m * p.y_cs + p.y_co;
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) +
                          (uint32_t)(buf * Cfg::kBufCols + blk * Cfg::kBlkCols);
      // fused head: this lane's half of the pre-head outputs for its pixel and its partner's
      const int hf = lane & 1;
      float hs[4], hp[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) hs[k] = hp[k] = fuse_head ? sbh[4 * hf + k] : 0.f;
#pragma unroll 1
      for (int c = co_beg; c < co_end; c += 16) {
        float d0[16], d1[16], d2[16], r[16], o16[16];
        // dx = 0, 1, 2 blocks (and the projection) in one TMEM read group
        if constexpr (RES) tmem_ld16x4(tb + c, tb + CO + c, tb + 2 * CO + c, tb + Cfg::kN + c, d0, d1, d2, r);
        else tmem_ld16x3(tb + c, tb + CO + c, tb + 2 * CO + c, d0, d1, d2);
#pragma unroll
        for (int j4 = 0; j4 < 16; j4 += 4) {
          float g4[4], b4[4], w0[4] = {0.f, 0.f, 0.f, 0.f}, w1[4] = {0.f, 0.f, 0.f, 0.f},
                                 w2[4] = {0.f, 0.f, 0.f, 0.f};
          lds4(sg + c + j4, g4);
          lds4(sb + c + j4, b4);
          if (rgb) {
            lds4(swp + c + j4, w0);
            lds4(swp + CO + c + j4, w1);
            lds4(swp + 2 * CO + c + j4, w2);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j4 + u;
            // lane-1 holds the left neighbour's dx=0 sum, lane+1 the right's dx=2 sum
            const float left = __shfl_up_sync(0xffffffffu, d0[j], 1);
            const float right = __shfl_down_sync(0xffffffffu, d2[j], 1);
            float z = fmaf(g4[u], left + d1[j] + right, b4[u]);
            if constexpr (RES) z += r[j];
            if (rgb) z += fmaf(v0, w0[u], fmaf(v1, w1[u], v2 * w2[u]));
            o16[j] = fmaxf(z, 0.f);
          }
        }
        if (writes && p.y) {
          uint32_t packed[8];
#pragma unroll
          for (int j = 0; j < 16; j += 2) packed[j / 2] = pack2(o16[j], o16[j + 1]);
          uint4* dst = reinterpret_cast<uint4*>(out + c);
          dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
        if (p.pool) {
          // valid columns are lanes 1..14 of a row group (tile origin even), so
          // an odd lane pairs with lane+1; lanes 0-15 / 16-31 hold rows 2k / 2k+1
          uint32_t pk[8];
          pool_pack(o16, true, pk);
          if (lane < 16 && (col & 1) && col < kXTW && ww < p.R) {
            uint4* dst = reinterpret_cast<uint4*>(
                p.pool + (((long long)img * (p.R >> 1) + (hh >> 1)) * (p.R >> 1) + (ww >> 1)) * p.pool_cs + c);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          }
        }
        if (fuse_head) {
#pragma unroll
          for (int j = 0; j < 16; ++j) prehead_pair(swh, c + j, o16[j], hf, hs, hp);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
      if (fuse_head) {
        // the TMEM buffer is released; the heads run on registers and shared memory
        float he[8], ho[8];
        prehead_pair_finish(hf, hs, hp, he, ho);
        if (img != th_img) {
          __syncwarp();
          const float* src = p.theta + (long long)img * p.ncls * kHeadParams;
          for (int i2 = lane; i2 < p.ncls * kHeadParams; i2 += 32)
            sth[(i2 / kHeadParams) * kThetaPad + i2 % kHeadParams] = src[i2];
          __syncwarp();
          th_img = img;
        }
        // the pair's pixels: this lane's and its partner's (halo lanes and
        // columns past R write nothing)
        const long long pix = (long long)hh * p.R + (ww < 0 ? 0 : ww);
        const long long pix_p = __shfl_xor_sync(0xffffffffu, pix, 1);
        const bool wr_p = __shfl_xor_sync(0xffffffffu, writes ? 1 : 0, 1) != 0;
        heads_pair(sth, p.ncls, RR, p.logits + (long long)(p.slot0 + img) * p.ncls * RR, hf, he, ho,
                   hf ? pix_p : pix, hf ? pix : pix_p, hf ? wr_p : writes, hf ? writes : wr_p);
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(Cfg::kTmemCols)
                 : "memory");
}

// ------------------------------------------------------------------ first layer
// conv3x3 of the normalised RGB tile (cin = 3) on the tensor cores.  No TMA
// box can read the uint8 canvas as an im2col operand, so the operand is built
// in two steps per 128-pixel tile (8 rows x 16 columns):
//   1. a TMA load of the tile's raw window, 10 canvas rows x 80 bytes starting
//      at the 16-byte boundary at or left of the window (the 18-pixel, 54-byte
//      window sits at byte offset 0..15 of each row; OOB rows read as zero);
//   2. builder thread r reads the nine bytes of each of its pixel's three
//      window rows as three aligned words (funnel-shifted into place) and
//      writes each byte u as the FP16 number 512 + u, whose bits are
//      0x6000 | 2u (FP16 spacing is 1/2 on [512, 1024)): two bytes become a
//      pair of halves with one byte permute and one multiply-add.  A tap
//      outside the tile takes 639.5 = 512 + 127.5 (bits 0x60FF), the value
//      at which the normalisation v = 2u/255 - 1 is zero.  The 64-byte K row
//      (the 27 operands, two constant 1s, zeros to 32; FP16 in every precision,
//      exact for 8-bit colour) is stored in the 64-byte-swizzled K-major
//      layout the MMA reads (16-byte chunk j of row r at chunk j ^ ((r >> 1) & 3)).
// Two FP16 MMAs (K = 16 each) per tile, N = cout.  The normalisation and the
// layer's norm ride in the weights: with A = 512 + u, v = (A - 639.5) 2/255,
// so g (w . v) + b = sum_k W_k A_k + B for W = g w 2/255 (entries 0..26,
// rounded to FP16) and B = b - 639.5 sum_k W_k over the rounded W (exact, so
// only the weight rounding remains), carried as an FP16 pair hi + lo in
// entries 27 and 28, whose operands are 1.  The accumulator already holds
// g * conv + b and the epilogue applies only the ReLU.  The epilogue stages
// each warp's 32 output pixels (two rows of 16) in shared memory, swizzled
// like the output tensor map, and writes them with one TMA store per warp and
// tile: whole 128-byte lines instead of 32 scattered 16-byte pieces per store.
//   warps 0-7  builders in two groups of four (group g builds the CTA's
//              tiles g, g + 2, ...: two tiles in flight), warp 8 MMA issuer +
//              TMEM owner, warps 9-16 epilogue in two groups of four taking
//              alternate tiles (lane quarters 1, 2, 3, 0 in each group),
//              warp 17 TMA producer of the raw windows.
__host__ __device__ constexpr uint32_t idesc_f16_ops(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}
// first-layer operand bits: FP16 512 + u for byte u, and 639.5 (v = 0) for a padding tap
constexpr uint32_t kFirstOp = 0x6000u, kFirstPad = 0x60FFu, kFirstOne = 0x3C00u;
constexpr int kFirstGroups = 2;                           // builder groups, 128 threads each
constexpr int kFirstBuilders = 128 * kFirstGroups;
constexpr int kFirstEpiGroups = 2;                         // epilogue warpgroups, alternate tiles
constexpr int kThreadsFirst = kFirstBuilders + 32 + 128 * kFirstEpiGroups + 32;
constexpr int kFirstMmaWarp = kFirstBuilders / 32, kFirstProducerWarp = kFirstMmaWarp + 1 + 4 * kFirstEpiGroups;
constexpr int kFirstStages = 8;
static_assert(kFirstStages % kFirstGroups == 0, "builder group g owns the ring slots s = g (mod groups)");
constexpr int kFirstRowBytes = 64;                        // 32 K values x 2 bytes
constexpr int kFirstStageBytes = kBM * kFirstRowBytes;    // 8 KB
constexpr int kRawW = 80, kRawH = kHTH + 2;               // raw window box (bytes x rows)
constexpr int kRawStageBytes = 1024;                      // 800 bytes used

template <int CO>
struct FirstCfg {
  static constexpr int kWBytes = CO * kFirstRowBytes;
  static constexpr int kBufCols = CO;
  static constexpr int kBufs = tmem_bufs(kBufCols);
  static constexpr int kTmemCols = tmem_alloc_cols(kBufs * kBufCols);
  static constexpr int kOutWarpBytes = 32 * CO * 2;       // one warp's staged pixels (two buffers each)
  static constexpr int kOutBytes = 4 * kFirstEpiGroups * 2 * kOutWarpBytes;
  static constexpr size_t kSmem =
      1024 + (size_t)kFirstStages * (kFirstStageBytes + kRawStageBytes) + kWBytes + kOutBytes + 2048;
};

// raw-window tensor maps of the batch's canvases (entry k for canvas cv.ptr[k])
struct CanvasMaps {
  CUtensorMap m[kMaxCanvases];
};

template <int CO>
__global__ void __launch_bounds__(kThreadsFirst, 1)
    k_conv_tc_first(const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CanvasMaps mapsC,
                    const __grid_constant__ CUtensorMap mapY, TCParams p) {
  using Cfg = FirstCfg<CO>;
  constexpr int ST = kFirstStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sRaw = sA + (size_t)ST * kFirstStageBytes;
  uint8_t* sW = sRaw + (size_t)ST * kRawStageBytes;
  uint8_t* sOut = sW + Cfg::kWBytes;               // 1024-aligned: the stages and sW are multiples of 1 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sOut + Cfg::kOutBytes);
  uint64_t* full = bars;                           // A stage built (4 builder warps)
  uint64_t* empty = bars + ST;                     // A stage consumed (MMA commit)
  uint64_t* rfull = bars + 2 * ST;                 // raw window landed (TMA)
  uint64_t* rempty = bars + 3 * ST;                // raw window read (4 builder warps)
  uint64_t* tfull = bars + 4 * ST;
  uint64_t* tempty = bars + 4 * ST + kMaxTmemBufs;
  uint64_t* drain = bars + 4 * ST + 2 * kMaxTmemBufs;
  uint64_t* wbar = drain + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wbar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), 4);
      mbar_init(smem_u32(&empty[s]), 1);
      mbar_init(smem_u32(&rfull[s]), 1);
      mbar_init(smem_u32(&rempty[s]), 4);
    }
    for (int b = 0; b < Cfg::kBufs; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), 4);
    }
    mbar_init(smem_u32(drain), 1);
    mbar_init(smem_u32(wbar), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == kFirstMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(Cfg::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == kFirstProducerWarp) {
    if (lane == 0) {
      // ---------------------------------------------------------------- raw-window producer
      StageRing ring;
      TileWalk tw;
      tw.init(p.R / kHTH, p.R / kHTW);
      int it = 0;
      for (; tw.t < p.n_tiles; tw.next(), ring.next(ST), ++it) {
        const int s = ring.s;
        if (ring.lapped && !mbar_wait(smem_u32(&rempty[s]), ring.ph ^ 1u, abort_flag, p.err)) break;
        const int sl = p.tiles3[3 * tw.img];
        const int y0 = p.tiles3[3 * tw.img + 1] + tw.ty * kHTH - 1;
        const int xb = (p.tiles3[3 * tw.img + 2] + tw.tx * kHTW - 1) * 3;
        const uint32_t fb = smem_u32(&rfull[s]);
        mbar_expect_tx(fb, kRawW * kRawH);
        tma_load_2d(smem_u32(sRaw + (size_t)s * kRawStageBytes), &mapsC.m[sl], fb, xb & ~15, y0);
      }
      for (int q = it - 1; q >= 0 && q >= it - ST; --q) mbar_drain(smem_u32(&rfull[q % ST]), (q / ST) & 1);
    }
  } else if (warp < kFirstMmaWarp) {
    // ------------------------------------------------------------------ builders
    const int grp = threadIdx.x / 128;               // builds the CTA's tiles grp, grp + groups, ...
    const int r = threadIdx.x % 128;                 // pixel row of the A tile
    const int rh = r / kHTW, rw = r % kHTW;          // its place in the 8 x 16 tile
    const int swz = (r >> 1) & 3;
    int s = grp;                                     // ring slot of the tile (ST is a multiple of the groups)
    uint32_t ph = 0;
    bool lapped = false;
    TileWalk tw;
    tw.init(p.R / kHTH, p.R / kHTW, (int)blockIdx.x + grp * (int)gridDim.x, kFirstGroups * (int)gridDim.x);
    int cimg = -1, cx0 = 0;                          // tile origin column of the current image
    for (; tw.t < p.n_tiles; tw.next()) {
      if (tw.img != cimg) {
        cimg = tw.img;
        cx0 = __ldg(p.tiles3 + 3 * tw.img + 2);
      }
      bool ok = !lapped || mbar_wait(smem_u32(&empty[s]), ph ^ 1u, abort_flag, p.err);
      ok = ok && mbar_wait(smem_u32(&rfull[s]), ph, abort_flag, p.err);
      if (!__all_sync(0xffffffffu, ok)) break;
      // byte of tap (dy, 0), channel 0 in its raw row: at most 15 + 45, so the
      // three words read per row end at byte 71 of the 80 loaded
      const int bb = (((cx0 + tw.tx * kHTW - 1) * 3) & 15) + rw * 3;
      const uint32_t* wrow = reinterpret_cast<const uint32_t*>(sRaw + (size_t)s * kRawStageBytes) + (bb >> 2);
      const uint32_t sh = (uint32_t)(bb & 3) * 8u;
      const int h_in = tw.ty * kHTH + rh - 1, w_in = tw.tx * kHTW + rw - 1;   // tile coords of tap (0, 0)
      // blocks whose 10 x 18 window lies inside the tile need no zero padding
      const bool inner = tw.ty > 0 && (tw.ty + 1) * kHTH < p.R && tw.tx > 0 && (tw.tx + 1) * kHTW < p.R;
      uint32_t wd[3][3];                             // bytes 0..8 of the three window rows
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const uint32_t* wp = wrow + (rh + dy) * (kRawW / 4);
        const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2];
        wd[dy][0] = __funnelshift_r(w0, w1, sh);
        wd[dy][1] = __funnelshift_r(w1, w2, sh);
        wd[dy][2] = __funnelshift_r(w2, w2, sh);
      }
      // K entry k = 9 dy + 3 dx + c is byte k % 9 of row k / 9; word i of the
      // row holds entries 2i and 2i + 1 (entry 27 and 28 are the constant 1s)
      uint32_t a16[16];
#pragma unroll
      for (int i = 0; i < 14; ++i) {
        const int k0 = 2 * i, k1 = 2 * i + 1;
        const uint32_t x0 = wd[k0 / 9][(k0 % 9) >> 2];
        const uint32_t b0 = (uint32_t)((k0 % 9) & 3);
        uint32_t pr;
        if (k1 == 27) {
          pr = __byte_perm(x0, 0u, b0 | 0x4440u);                      // [u0, 0, 0, 0]
        } else if (k0 / 9 == k1 / 9 && (k0 % 9) >> 2 == (k1 % 9) >> 2) {
          const uint32_t b1 = (uint32_t)((k1 % 9) & 3);
          pr = __byte_perm(x0, 0u, b0 | 0x4040u | (b1 << 8));          // [u0, 0, u1, 0]
        } else {
          const uint32_t b1 = (uint32_t)((k1 % 9) & 3) + 4u;
          pr = __byte_perm(x0, wd[k1 / 9][(k1 % 9) >> 2], b0 | (b1 << 8)) & 0x00FF00FFu;
        }
        uint32_t h = pr * 2u + (kFirstOp | kFirstOp << 16);            // halves 512 + u
        if (k1 == 27) h = (h & 0xFFFFu) | kFirstOne << 16;
        a16[i] = h;
      }
      if (!inner) {
        // zero padding: taps outside the tile take the operand of v = 0
        bool yin[3], xin[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          yin[d] = h_in + d >= 0 && h_in + d < p.R;
          xin[d] = w_in + d >= 0 && w_in + d < p.R;
        }
#pragma unroll
        for (int i = 0; i < 14; ++i) {
          const int k0 = 2 * i, k1 = 2 * i + 1;
          uint32_t m = yin[k0 / 9] && xin[(k0 % 9) / 3] ? 0u : 0xFFFFu;
          if (k1 != 27) m |= yin[k1 / 9] && xin[(k1 % 9) / 3] ? 0u : 0xFFFF0000u;
          a16[i] = (a16[i] & ~m) | ((kFirstPad | kFirstPad << 16) & m);
        }
      }
      a16[14] = kFirstOne;                           // entry 28 = 1 (operand of the shift's low half)
      a16[15] = 0u;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&rempty[s]));
      uint8_t* row = sA + (size_t)s * kFirstStageBytes + r * kFirstRowBytes;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        *reinterpret_cast<uint4*>(row + ((j ^ swz) << 4)) =
            make_uint4(a16[4 * j], a16[4 * j + 1], a16[4 * j + 2], a16[4 * j + 3]);
      // make this thread's generic-proxy stores visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&full[s]));
      s += kFirstGroups;
      if (s >= ST) {
        s -= ST;
        ph ^= 1u;
        lapped = true;
      }
    }
  } else if (warp == kFirstMmaWarp) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuer
      const uint32_t wb = smem_u32(wbar);
      mbar_expect_tx(wb, (uint32_t)Cfg::kWBytes);
      tma_load_2d(smem_u32(sW), &mapB, wb, 0, 0);
      constexpr uint32_t idesc = idesc_f16_ops(CO);
      const uint64_t a_desc0 = smem_desc(smem_u32(sA), kFirstRowBytes);
      const uint64_t b_desc = smem_desc(smem_u32(sW), kFirstRowBytes);
      bool ok = mbar_wait(wb, 0, abort_flag, p.err);
      int tcount = 0;
      StageRing ring;
      for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x, ++tcount, ring.next(ST)) {
        const int buf = tcount % Cfg::kBufs, use = tcount / Cfg::kBufs;
        if (use >= 1 && !mbar_wait(smem_u32(&tempty[buf]), (use - 1) & 1, abort_flag, p.err)) break;
        const int s = ring.s;
        if (!mbar_wait(smem_u32(&full[s]), ring.ph, abort_flag, p.err)) break;
        tc_fence_after();
        const uint32_t acc = tmem_base + (uint32_t)(buf * Cfg::kBufCols);
        const uint64_t ad = a_desc0 + (uint64_t)((s * kFirstStageBytes) >> 4);
        mma_bf16(acc, ad, b_desc, idesc, 0u);
        mma_bf16(acc, ad + 2, b_desc + 2, idesc, 1u);
        mma_commit(smem_u32(&empty[s]));
        mma_commit(smem_u32(&tfull[buf]));
      }
      mma_commit(smem_u32(drain));
      mbar_drain(smem_u32(drain), 0);
      mbar_drain(wb, 0);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    // two warpgroups take alternate tiles, so one group's TMEM read and stores
    // overlap the other's; warp w of a group reads lane quarter w % 4, i.e.
    // pixels 32 q .. 32 q + 31 of the tile: tile rows 2q, 2q + 1, which is the
    // output box {CO channels, 16 columns, 2 rows} with lane = staged row
    const int q = warp & 3;
    const int ew = warp - kFirstMmaWarp - 1;
    const int grp = ew / 4;
    // staged row = lane, swizzled like the output map (64-byte rows: chunk
    // j ^ ((row >> 1) & 3); 128-byte rows: chunk j ^ (row & 7))
    const int osw = CO == 32 ? (lane >> 1) & 3 : lane & 7;
    uint8_t* stg0 = sOut + (size_t)ew * 2 * Cfg::kOutWarpBytes;
    int tcount = 0, lt = 0;
    TileWalk tw;
    tw.init(p.R / kHTH, p.R / kHTW);
    for (; tw.t < p.n_tiles; tw.next(), ++tcount) {
      if ((tcount & 1) != grp) continue;
      const int buf = tcount % Cfg::kBufs, use = tcount / Cfg::kBufs;
      const bool ok = mbar_wait(smem_u32(&tfull[buf]), use & 1, abort_flag, p.err);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      // staging buffer lt & 1: the store issued from it two tiles ago has read it
      if (lane == 0) bulk_wait_read1();
      __syncwarp();
      uint8_t* srow = stg0 + (size_t)(lt & 1) * Cfg::kOutWarpBytes + lane * (CO * 2);
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * Cfg::kBufCols);
#pragma unroll
      for (int c = 0; c < CO; c += 32) {
        float a2[2][16];
        tmem_ld16x2(tb + c, tb + c + 16, a2[0], a2[1]);   // 32 columns, one wait
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cc = c + 16 * h;
          const float* a = a2[h];
          uint32_t packed[8];
#pragma unroll
          for (int j = 0; j < 16; j += 2) packed[j / 2] = pack2(fmaxf(a[j], 0.f), fmaxf(a[j + 1], 0.f));
          const int j0 = cc / 8;
          *reinterpret_cast<uint4*>(srow + ((j0 ^ osw) << 4)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          *reinterpret_cast<uint4*>(srow + (((j0 + 1) ^ osw) << 4)) =
              make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
      }
      tc_fence_before();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&tempty[buf]));
        tma_store_4d(&mapY, smem_u32(stg0 + (size_t)(lt & 1) * Cfg::kOutWarpBytes), 0, tw.tx * kHTW,
                     tw.ty * kHTH + 2 * q, tw.img);
        bulk_commit();
      }
      ++lt;
    }
    // the output must be in global memory before the kernel ends
    if (lane == 0) bulk_wait_all();
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kFirstMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(Cfg::kTmemCols)
                 : "memory");
}

// ------------------------------------------------------------------ host side
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

// NHWC activation box: {CK channels, bw pixels, bh rows, 1 image}; eb bytes
// per element (2: BF16 / FP16, 1: E4M3 bytes)
bool map_act(CUtensorMap* m, const void* base, int channels, int cs, int co, int R, int B, int CK,
             int eb = 2) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  const char* ptr = static_cast<const char*>(base) + (size_t)co * eb;
  cuuint64_t dims[4] = {(cuuint64_t)channels, (cuuint64_t)R, (cuuint64_t)R, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)cs * eb, (cuuint64_t)R * cs * eb, (cuuint64_t)R * R * cs * eb};
  const int bw = R < kBM ? R : kBM;
  cuuint32_t box[4] = {(cuuint32_t)CK, (cuuint32_t)bw, (cuuint32_t)(kBM / bw), 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, eb == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                   const_cast<char*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CK * eb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// NHWC activation box of bw x bh pixels (small-N variant: 16 x 10 or 16 x 8)
bool map_act_box(CUtensorMap* m, const void* base, int channels, int cs, int co, int R, int B, int CK,
                 int bw, int bh) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  const char* ptr = static_cast<const char*>(base) + (size_t)co * 2;
  cuuint64_t dims[4] = {(cuuint64_t)channels, (cuuint64_t)R, (cuuint64_t)R, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)cs * 2, (cuuint64_t)R * cs * 2, (cuuint64_t)R * R * cs * 2};
  cuuint32_t box[4] = {(cuuint32_t)CK, (cuuint32_t)bw, (cuuint32_t)bh, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<char*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// K-major weights [rows = cout][K]: box {CK, BN}; eb bytes per element
bool map_w(CUtensorMap* m, const void* base, int K, int cout, int BN, int CK, int eb = 2) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)cout};
  cuuint64_t strides[1] = {(cuuint64_t)K * eb};
  cuuint32_t box[2] = {(cuuint32_t)CK, (cuuint32_t)BN};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, eb == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CK * eb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

template <int BN, int CK, bool RES, bool PAIR = false, bool F8 = false>
cudaError_t launch_t(const ConvArgs& a, cudaStream_t st) {
  using Cfg = TCCfg<BN, CK, RES, PAIR, F8>;
  CUtensorMap mA, mB, mA2, mB2;
  if (!map_act(&mA, a.x, a.cin, a.x_cs, a.x_co, a.R, a.B, CK, Cfg::kEB)) return cudaErrorInvalidValue;
  if (!map_w(&mB, a.w.w_bf16, 9 * a.cin, a.cout, Cfg::kBRows, CK, Cfg::kEB)) return cudaErrorInvalidValue;
  if (RES) {
    if (!map_act(&mA2, a.r, a.cr, a.r_cs, a.r_co, a.R, a.B, CK)) return cudaErrorInvalidValue;
    if (!map_w(&mB2, a.w.wp_bf16, a.cr, a.cout, Cfg::kBRows, CK)) return cudaErrorInvalidValue;
  } else {
    mA2 = mA;
    mB2 = mB;
  }
  TCParams p{};
  p.B = a.B; p.R = a.R; p.cin = a.cin; p.cout = a.cout; p.cr = RES ? a.cr : 0;
  p.res_mode = a.res_mode;
  p.n_tiles_m = (int)((long long)a.B * a.R * a.R / kBM);
  p.n_tiles_n = a.cout / BN;
  p.n_tiles = p.n_tiles_m * p.n_tiles_n;
  p.k_main = 9 * (a.cin / CK);
  p.k_res = RES ? a.cr / CK : 0;
  p.gamma = a.w.gamma;
  p.beta = a.w.beta;
  p.wp_rgb = a.w.wp_f32;
  p.cv = a.cv;
  p.tiles3 = a.tiles3;
  p.y = static_cast<__nv_bfloat16*>(a.y);
  p.y_cs = a.y_cs;
  p.y_co = a.y_co;
  p.err = a.err;
  if (a.pool || a.head_theta || !a.y) return cudaErrorInvalidValue;   // no fused outputs here
  auto kern = k_conv_tc<BN, CK, RES, PAIR, F8>;
  static bool attr_set = false;
  static int max_pairs = 0;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    if (e != cudaSuccess) return e;
    if (PAIR) {
      cudaLaunchConfig_t q = {};
      q.gridDim = dim3(2 * (num_sms() / 2));
      q.blockDim = dim3(kThreadsTC);
      q.dynamicSmemBytes = Cfg::kSmem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      q.attrs = at;
      q.numAttrs = 1;
      e = cudaOccupancyMaxActiveClusters(&max_pairs, kern, &q);
      if (e != cudaSuccess || max_pairs < 1) return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
    }
    attr_set = true;
  }
  if (!PAIR) {
    int grid = p.n_tiles < num_sms() ? p.n_tiles : num_sms();
    kern<<<grid, kThreadsTC, Cfg::kSmem, st>>>(mA, mB, mA2, mB2, p);
    return cudaGetLastError();
  }
  // pairs take M tiles 2 a, 2 a + 1 of one N tile: the M tile count must be even
  if (p.n_tiles_m % 2) return cudaErrorInvalidValue;
  const int pairs = p.n_tiles / 2 < max_pairs ? p.n_tiles / 2 : max_pairs;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(kThreadsTC);
  cfg.dynamicSmemBytes = Cfg::kSmem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, mA, mB, mA2, mB2, p);
  if (e != cudaSuccess) cudaGetLastError();   // a refused launch leaves no sticky state behind
  return e;
}

constexpr int kHaloSmemMax = 227 * 1024;
constexpr int kHaloSmemExtra = 3072;   // barriers, gamma/beta, alignment slack
// fused head: wh[8][64] + bh[8] + a 2-class theta copy per epilogue warp
constexpr int kHeadSmem = (kHeadCh * 64 + kHeadCh + kEpiWarps * 2 * kThetaPad) * 4 + 16;

// copy the optional fused outputs of a launch into the kernel parameters
void set_fused(const ConvArgs& a, TCParams& p, bool head_ok) {
  p.pool = static_cast<__nv_bfloat16*>(a.pool);
  p.pool_cs = a.pool_cs;
  if (head_ok && a.head_theta) {
    p.theta = a.head_theta;
    p.wh = a.head_wh;
    p.bh = a.head_bh;
    p.logits = a.head_logits;
    p.slot0 = a.head_slot0;
    p.ncls = a.head_ncls;
  }
}

// slots of the small-N variant for a layer, channel chunk and blocks per tile (0: does not fit)
int halo_stages(int cin, int cout, int cr, int ck, int mb = 1) {
  if (cin % ck || cr % ck) return 0;
  const long long wbytes = (long long)(9 * (cin / ck) + cr / ck) * cout * ck * 2;
  const long long stage = 3LL * (kHTH * mb + 2) * kHTW * ck * 2;
  long long st = (kHaloSmemMax - wbytes - kHaloSmemExtra) / stage;
  return st < 2 ? 0 : (int)(st > 8 ? 8 : st);
}

bool halo_ok(int R, int cout, int cin, int cr) {
  if (R < 16 || R % 16 || (cout != 32 && cout != 64)) return false;
  return halo_stages(cin, cout, cr, 32) >= 2;
}

template <int BN, int CK, bool RES, int MB, bool PAIR = false>
cudaError_t launch_halo(const ConvArgs& a, cudaStream_t st, int stages) {
  using Cfg = HaloCfg<BN, CK, RES, MB, PAIR>;
  CUtensorMap mA, mB, mA2, mB2;
  if (a.R % (kHTH * MB)) return cudaErrorInvalidValue;
  if (!map_act_box(&mA, a.x, a.cin, a.x_cs, a.x_co, a.R, a.B, CK, kHTW, Cfg::kBoxRows)) return cudaErrorInvalidValue;
  if (!map_w(&mB, a.w.w_bf16, 9 * a.cin, a.cout, Cfg::kWRows, CK)) return cudaErrorInvalidValue;
  if (RES) {
    if (!map_act_box(&mA2, a.r, a.cr, a.r_cs, a.r_co, a.R, a.B, CK, kHTW, kHTH * MB)) return cudaErrorInvalidValue;
    if (!map_w(&mB2, a.w.wp_bf16, a.cr, a.cout, Cfg::kWRows, CK)) return cudaErrorInvalidValue;
  } else {
    mA2 = mA;
    mB2 = mB;
  }
  HaloParams hp{};
  TCParams& p = hp.t;
  p.B = a.B; p.R = a.R; p.cin = a.cin; p.cout = a.cout; p.cr = RES ? a.cr : 0;
  p.res_mode = a.res_mode;
  hp.tiles_w = a.R / kHTW;
  hp.tiles_per_img = (a.R / (kHTH * MB)) * hp.tiles_w;
  p.n_tiles_m = a.B * hp.tiles_per_img;
  p.n_tiles_n = 1;
  p.n_tiles = p.n_tiles_m;
  p.k_main = a.cin / CK;
  hp.res_chunks = RES ? a.cr / CK : 0;
  p.k_res = (hp.res_chunks + 2) / 3;
  hp.cpt = a.cin / CK;
  hp.n_wtiles = 9 * hp.cpt + hp.res_chunks;
  // stages hold up to a tile's slots while at least three stages stay in flight
  hp.group = max(1, min(p.k_main + p.k_res, stages / 3));
  stages /= hp.group;
  hp.stages = stages;
  p.gamma = a.w.gamma;
  p.beta = a.w.beta;
  p.wp_rgb = a.w.wp_f32;
  p.cv = a.cv;
  p.tiles3 = a.tiles3;
  p.y = static_cast<__nv_bfloat16*>(a.y);
  p.y_cs = a.y_cs;
  p.y_co = a.y_co;
  p.err = a.err;
  const bool head = a.head_theta != nullptr;
  if (head && (a.head_ncls < 1 || a.head_ncls > 2 || !a.head_wh || !a.head_bh || !a.head_logits))
    return cudaErrorInvalidValue;
  if (!head && !a.y) return cudaErrorInvalidValue;
  set_fused(a, p, true);
  const size_t fixed = (size_t)hp.n_wtiles * Cfg::kWTileBytes + kHaloSmemExtra + (head ? kHeadSmem : 0);
  const size_t stage_bytes = (size_t)hp.group * Cfg::kStageBytes;
  if (head && fixed + (size_t)stages * stage_bytes > (size_t)kHaloSmemMax)
    stages = (int)(((size_t)kHaloSmemMax - fixed) / stage_bytes);   // room for the head's arrays
  if (stages < 2) return cudaErrorInvalidValue;
  hp.stages = stages;
  const size_t smem = fixed + (size_t)stages * stage_bytes;
  if (smem > (size_t)kHaloSmemMax) return cudaErrorInvalidValue;
  auto kern = k_conv_tc_halo<BN, CK, RES, MB, PAIR>;
  static bool attr_set = false;
  static int max_pairs = 0;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kHaloSmemMax);
    if (e != cudaSuccess) return e;
    if (PAIR) {
      cudaLaunchConfig_t q = {};
      q.gridDim = dim3(2 * (num_sms() / 2));
      q.blockDim = dim3(kThreadsTC);
      q.dynamicSmemBytes = kHaloSmemMax;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      q.attrs = at;
      q.numAttrs = 1;
      e = cudaOccupancyMaxActiveClusters(&max_pairs, kern, &q);
      if (e != cudaSuccess || max_pairs < 1) return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
    }
    attr_set = true;
  }
  if (!PAIR) {
    int grid = p.n_tiles < num_sms() ? p.n_tiles : num_sms();
    kern<<<grid, kThreadsTC, smem, st>>>(mA, mB, mA2, mB2, hp);
    return cudaGetLastError();
  }
  // pairs: CTA 0 of cluster k takes tiles 2k, 2k + grid, ..., CTA 1 the next
  // ones; both need the same count, so the tile count must be even
  if (p.n_tiles % 2) return cudaErrorInvalidValue;
  int pairs = p.n_tiles / 2 < max_pairs ? p.n_tiles / 2 : max_pairs;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(kThreadsTC);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, mA, mB, mA2, mB2, hp);
  if (e != cudaSuccess) cudaGetLastError();   // a refused launch leaves no sticky state behind
  return e;
}

// dx-in-N variant: resident weights + one 10 x 16 box per stage
int dxn_wbytes(int cin, int cout, int cr, int ck) { return (9 * (cin / ck) + cr / ck) * cout * ck * 2; }
int dxn_stages(int cin, int cout, int cr, int ck, int mb = 1) {
  if (cin % ck || cr % ck) return 0;
  const long long st = (kHaloSmemMax - (long long)dxn_wbytes(cin, cout, cr, ck) - kHaloSmemExtra) /
                       ((long long)(kHTH * mb + 2) * kHTW * ck * 2);
  return st < 2 ? 0 : (int)(st > 12 ? 12 : st);
}
bool dxn_ok(int R, int cout, int cin, int cr) {
  if (R < 16 || R % kHTH || (cout != 32 && cout != 64)) return false;
  return dxn_stages(cin, cout, cr, 32) >= 2;
}

template <int CO, int CK, bool RES, int MB>
cudaError_t launch_dxn(const ConvArgs& a, cudaStream_t st, int stages) {
  using Cfg = DxnCfg<CO, CK, RES, MB>;
  CUtensorMap mA, mB, mA2, mB2;
  if (a.R % (kHTH * MB)) return cudaErrorInvalidValue;
  if (!map_act_box(&mA, a.x, a.cin, a.x_cs, a.x_co, a.R, a.B, CK, kHTW, Cfg::kBoxRows)) return cudaErrorInvalidValue;
  if (!map_w(&mB, a.w.w_bf16, 9 * a.cin, a.cout, CO, CK)) return cudaErrorInvalidValue;
  if (RES) {
    if (!map_act_box(&mA2, a.r, a.cr, a.r_cs, a.r_co, a.R, a.B, CK, kHTW, kHTH * MB)) return cudaErrorInvalidValue;
    if (!map_w(&mB2, a.w.wp_bf16, a.cr, a.cout, CO, CK)) return cudaErrorInvalidValue;
  } else {
    mA2 = mA;
    mB2 = mB;
  }
  DxnParams hp{};
  TCParams& p = hp.t;
  p.B = a.B; p.R = a.R; p.cin = a.cin; p.cout = a.cout; p.cr = RES ? a.cr : 0;
  p.res_mode = a.res_mode;
  hp.tiles_w = (a.R + kXTW - 1) / kXTW;
  hp.tiles_per_img = (a.R / (kHTH * MB)) * hp.tiles_w;
  p.n_tiles_m = a.B * hp.tiles_per_img;
  p.n_tiles_n = 1;
  p.n_tiles = p.n_tiles_m;
  hp.cpt = a.cin / CK;
  hp.res_chunks = RES ? a.cr / CK : 0;
  // a tile's slots (main chunks, then projection chunks) are grouped into
  // stages of up to the whole tile, keeping at least three stages in flight:
  // fewer waits and commits per MMA
  const int slots = hp.cpt + hp.res_chunks;
  hp.cps = max(1, min(slots, stages / 3));
  p.k_main = slots;                   // the loops walk slots 0 .. slots-1 in steps of cps
  p.k_res = 0;
  stages /= hp.cps;
  hp.wbytes = dxn_wbytes(a.cin, a.cout, RES ? a.cr : 0, CK);
  p.gamma = a.w.gamma;
  p.beta = a.w.beta;
  p.wp_rgb = a.w.wp_f32;
  p.cv = a.cv;
  p.tiles3 = a.tiles3;
  p.y = static_cast<__nv_bfloat16*>(a.y);
  p.y_cs = a.y_cs;
  p.y_co = a.y_co;
  p.err = a.err;
  // the fused head needs a thread to hold all channels of its pixel: with one
  // block per tile the two epilogue warpgroups then take alternate tiles
  const bool head = a.head_theta != nullptr;
  if (head && (a.head_ncls < 1 || a.head_ncls > 2 || !a.head_wh || !a.head_bh || !a.head_logits ||
               (MB == 1 && Cfg::kBufs % 2)))
    return cudaErrorInvalidValue;
  if (!head && !a.y) return cudaErrorInvalidValue;
  set_fused(a, p, true);
  const size_t fixed = (size_t)hp.wbytes + kHaloSmemExtra + (head ? kHeadSmem : 0);
  const size_t stage_bytes = (size_t)hp.cps * Cfg::kStageBytes;
  if (head && fixed + (size_t)stages * stage_bytes > (size_t)kHaloSmemMax)
    stages = (int)(((size_t)kHaloSmemMax - fixed) / stage_bytes);   // room for the head's arrays
  hp.stages = stages;
  const size_t smem = fixed + (size_t)stages * stage_bytes;
  if (stages < 2 || smem > (size_t)kHaloSmemMax) return cudaErrorInvalidValue;
  auto kern = k_conv_tc_dxn<CO, CK, RES, MB>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kHaloSmemMax);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int grid = p.n_tiles < num_sms() ? p.n_tiles : num_sms();
  kern<<<grid, kThreadsTC, smem, st>>>(mA, mB, mA2, mB2, hp);
  return cudaGetLastError();
}


// the uint8 canvas as a 2D byte tensor {row bytes, rows}: raw-window boxes
bool map_canvas(CUtensorMap* m, const uint8_t* canvas, long long stride, int canvas_h) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)stride, (cuuint64_t)canvas_h};
  cuuint64_t strides[1] = {(cuuint64_t)stride};
  cuuint32_t box[2] = {(cuuint32_t)kRawW, (cuuint32_t)kRawH};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(canvas), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// first-layer output as a store target: {CO channels, R, R, B} at channel
// offset co of rows cs channels long; box {CO, 16 columns, 2 rows, 1 image},
// swizzled like the epilogue's staging (64-byte rows for CO = 32, 128 for 64)
bool map_out_first(CUtensorMap* m, void* base, int CO, int cs, int co, int R, int B) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  char* ptr = static_cast<char*>(base) + (size_t)co * 2;
  cuuint64_t dims[4] = {(cuuint64_t)CO, (cuuint64_t)R, (cuuint64_t)R, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)cs * 2, (cuuint64_t)R * cs * 2, (cuuint64_t)R * R * cs * 2};
  cuuint32_t box[4] = {(cuuint32_t)CO, (cuuint32_t)kHTW, 2, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, ptr, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CO == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int CO>
cudaError_t launch_first(const ConvArgs& a, cudaStream_t st) {
  using Cfg = FirstCfg<CO>;
  CUtensorMap mB, mY;
  CanvasMaps mC;
  if (!map_w(&mB, a.w.w_bf16, 32, a.cout, CO, 32)) return cudaErrorInvalidValue;
  if (!map_out_first(&mY, a.y, CO, a.y_cs, a.y_co, a.R, a.B)) return cudaErrorInvalidValue;
  for (int k = 0; k < kMaxCanvases; ++k) {
    if (k > 0 && a.cv.ptr[k] == a.cv.ptr[k - 1] && a.cv.stride[k] == a.cv.stride[k - 1] &&
        a.cv.rows[k] == a.cv.rows[k - 1]) {
      mC.m[k] = mC.m[k - 1];
    } else if (a.cv.ptr[k]) {
      if (!map_canvas(&mC.m[k], a.cv.ptr[k], a.cv.stride[k], a.cv.rows[k])) return cudaErrorInvalidValue;
    } else {
      mC.m[k] = mC.m[0];     // unused entry: never indexed by a tile of this batch
    }
  }
  TCParams p{};
  p.B = a.B; p.R = a.R; p.cin = 3; p.cout = a.cout;
  p.n_tiles_m = a.B * (a.R / kHTH) * (a.R / kHTW);
  p.n_tiles_n = 1;
  p.n_tiles = p.n_tiles_m;
  p.gamma = a.w.gamma;
  p.beta = a.w.beta;
  p.cv = a.cv;
  p.tiles3 = a.tiles3;
  p.y = static_cast<__nv_bfloat16*>(a.y);
  p.y_cs = a.y_cs;
  p.y_co = a.y_co;
  p.err = a.err;
  auto kern = k_conv_tc_first<CO>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int grid = p.n_tiles < num_sms() ? p.n_tiles : num_sms();
  kern<<<grid, kThreadsFirst, Cfg::kSmem, st>>>(mB, mC, mY, p);
  return cudaGetLastError();
}

int pick_bn(int cout, bool res) {
  const int cap = res ? 128 : 256;
  return cout < cap ? cout : cap;
}

}  // namespace

#if !OMNI_TC_F16
bool conv_tc_supported(int R, int cin, int cout, int cr) {
  if (cin % 32 == 0 && cr % 32 == 0 && halo_ok(R, cout, cin, cr)) return true;
  if (cin % 32 == 0 && cr % 32 == 0 && R >= 64 && dxn_ok(R, cout, cin, cr)) return true;
  if (cout > 512) return false;
  if (!(R == 16 || R == 32 || R == 64 || (R >= 128 && R % 128 == 0))) return false;
  if (cin % 32 || cr % 32 || cout % 32) return false;
  const int bn = pick_bn(cout, cr > 0);
  return bn % 32 == 0 && cout % bn == 0;
}
#endif

namespace {
cudaError_t check_tc_args(const ConvArgs& a, int cr) {
  if (a.res_mode == RES_RGB && !a.w.wp_f32) return cudaErrorInvalidValue;
  if ((a.x_co % 8) || (a.x_cs % 8) || (a.y_co % 8) || (a.y_cs % 8)) return cudaErrorInvalidValue;
  if (cr && ((a.r_co % 8) || (a.r_cs % 8))) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.y) |
       reinterpret_cast<uintptr_t>(a.w.w_bf16) | (cr ? reinterpret_cast<uintptr_t>(a.r) |
                                                     reinterpret_cast<uintptr_t>(a.w.wp_bf16) : 0)) % 16)
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

bool pertap_ok(int R, int cin, int cout, int cr, int bn, int ck) {
  if (!(R == 16 || R == 32 || R == 64 || (R >= 128 && R % 128 == 0))) return false;
  if (cin % ck || cr % ck || bn > cout || cout % bn || cout > 512) return false;
  if (cr > 0 && bn > 128) return false;
  return bn == 32 || bn == 64 || bn == 128 || bn == 256;
}
}  // namespace

#if !OMNI_TC_F16
int tc_candidates(int R, int cin, int cout, int cr, TcConfig* out, int max) {
  int n = 0;
  if (dxn_ok(R, cout, cin, cr)) {
    for (int ck = 32; ck <= 64; ck *= 2) {
      const int stg = dxn_stages(cin, cout, cr, ck);
      if (stg >= 2 && n < max) out[n++] = TcConfig{2, cout, ck, stg};
    }
    const int stg2 = dxn_stages(cin, cout, cr, 32, 2);
    if (cout == 32 && R % 16 == 0 && stg2 >= 2 && n < max) out[n++] = TcConfig{4, 32, 32, stg2};
  }
  // kind 4 per 32-output-channel slice (weights of a slice resident)
  if (cout >= 64 && cout <= 256 && cout % 32 == 0 && R % 16 == 0 && dxn_ok(R, 32, cin, cr)) {
    const int stg = dxn_stages(cin, 32, cr, 32, 2);
    if (stg >= 2 && n < max) out[n++] = TcConfig{7, 32, 32, stg};
  }
  if (halo_ok(R, cout, cin, cr)) {
    for (int ck = 32; ck <= 64; ck *= 2) {
      const int stg = halo_stages(cin, cout, cr, ck);
      if (stg >= 2 && n < max) out[n++] = TcConfig{1, cout, ck, stg};
    }
    const int stg2 = halo_stages(cin, cout, cr, 32, 2);
    if (stg2 >= 2 && n < max) out[n++] = TcConfig{3, cout, 32, stg2};
    if (stg2 >= 2 && n < max) out[n++] = TcConfig{6, cout, 32, stg2};
  }
  for (int bn = 32; bn <= 256; bn *= 2)
    for (int ck = 32; ck <= 64; ck *= 2)
      if (pertap_ok(R, cin, cout, cr, bn, ck) && n < max) out[n++] = TcConfig{0, bn, ck, 0};
  // per-tap on CTA pairs, for the wide N tiles whose B traffic it halves
  for (int bn = 128; bn <= 256; bn *= 2)
    if (pertap_ok(R, cin, cout, cr, bn, 64) && (long long)R * R % (2 * kBM) == 0 && n < max)
      out[n++] = TcConfig{8, bn, 64, 0};
  return n;
}

bool tc_fuses_pool(const TcConfig& c) { return c.kind >= 1 && c.kind <= 6 && c.kind != 5; }

bool tc_fuses_head(const TcConfig& c, int cout, int ncls) {
  return ((c.kind == 1 || c.kind == 2 || c.kind == 3 || c.kind == 6) && (cout == 32 || cout == 64) ||
          (c.kind == 4 && cout == 32)) &&
         ncls >= 1 && ncls <= 2;
}

TcConfig tc_default(int R, int cin, int cout, int cr) {
  // measured: the dx-in-N kernel wins when a tile carries at least 64 input
  // channels of work; with 32 its epilogue dominates and the 3-box kernel wins
  if (R >= 64 && cin >= 64 && dxn_ok(R, cout, cin, cr)) {
    int ck = 32, stg = dxn_stages(cin, cout, cr, 32);
    const int stg64 = dxn_stages(cin, cout, cr, 64);
    if (stg64 >= 4) { ck = 64; stg = stg64; }
    const int stg2 = dxn_stages(cin, cout, cr, 32, 2);
    if (cout == 32 && ck == 32 && R % 16 == 0 && stg2 >= 4) return TcConfig{4, 32, 32, stg2};
    return TcConfig{2, cout, ck, stg};
  }
  if (halo_ok(R, cout, cin, cr)) {
    int ck = 32, stg = halo_stages(cin, cout, cr, 32);
    const int stg64 = halo_stages(cin, cout, cr, 64);
    if (stg64 >= 3) { ck = 64; stg = stg64; }
    // 32-channel chunks: two blocks per tile halve the per-tile synchronisation
    const int stg2 = halo_stages(cin, cout, cr, 32, 2);
    if (ck == 32 && stg2 >= 2) return TcConfig{3, cout, 32, stg2};
    return TcConfig{1, cout, ck, stg};
  }
  const bool res = cr > 0;
  return TcConfig{0, pick_bn(cout, res), (cin % 64 == 0 && (!res || cr % 64 == 0)) ? 64 : 32, 0};
}

#endif

#if OMNI_TC_F16
cudaError_t launch_conv_tc_cfg_f16(const ConvArgs& a, const TcConfig& c, cudaStream_t st) {
#else
cudaError_t launch_conv_tc_cfg_bf16(const ConvArgs& a, const TcConfig& c, cudaStream_t st) {
#endif
  const int cr = a.res_mode == RES_TENSOR ? a.cr : 0;
  cudaError_t e = check_tc_args(a, cr);
  if (e != cudaSuccess) return e;
  const bool res = cr > 0;
  if (c.kind == 2) {
    if (!dxn_ok(a.R, a.cout, a.cin, cr) || c.bn != a.cout || c.stages < 2 ||
        c.stages > dxn_stages(a.cin, a.cout, cr, c.ck))
      return cudaErrorInvalidValue;
#define OMNI_DXN(CO_, CK_, RES_) \
    if (c.bn == CO_ && c.ck == CK_ && res == RES_) return launch_dxn<CO_, CK_, RES_, 1>(a, st, c.stages);
    OMNI_DXN(32, 32, false) OMNI_DXN(32, 32, true) OMNI_DXN(32, 64, false) OMNI_DXN(32, 64, true)
    OMNI_DXN(64, 32, false) OMNI_DXN(64, 32, true) OMNI_DXN(64, 64, false) OMNI_DXN(64, 64, true)
#undef OMNI_DXN
    return cudaErrorInvalidValue;
  }
  if (c.kind == 7) {
    // one kind-4 launch per 32 output channels: a slice's weight rows, gamma,
    // beta and projection rows are contiguous; its output starts at channel
    // y_co + 32 h.  No fused pool / head / RGB projection (they need every
    // channel of a pixel, or a strided weight layout).
    if (a.res_mode == RES_RGB || a.pool || a.head_theta || a.cout < 64 || a.cout > 256 || a.cout % 32 ||
        a.R % 16 || c.bn != 32 || c.ck != 32 || !dxn_ok(a.R, 32, a.cin, cr) || c.stages < 2 ||
        c.stages > dxn_stages(a.cin, 32, cr, 32, 2))
      return cudaErrorInvalidValue;
    for (int h = 0; h < a.cout / 32; ++h) {
      ConvArgs sl = a;
      sl.cout = 32;
      sl.w.w_bf16 = a.w.w_bf16 + (size_t)h * 32 * 9 * a.cin;
      sl.w.gamma = a.w.gamma + 32 * h;
      sl.w.beta = a.w.beta + 32 * h;
      if (res) sl.w.wp_bf16 = a.w.wp_bf16 + (size_t)h * 32 * cr;
      sl.y_co = a.y_co + 32 * h;
      cudaError_t e = res ? launch_dxn<32, 32, true, 2>(sl, st, c.stages) : launch_dxn<32, 32, false, 2>(sl, st, c.stages);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (c.kind == 4) {
    // two blocks per tile: cout 32 only (TMEM holds two buffers of 2 x (96 + 32) columns)
    if (!dxn_ok(a.R, a.cout, a.cin, cr) || a.cout != 32 || c.bn != 32 || c.ck != 32 || a.R % 16 ||
        c.stages < 2 || c.stages > dxn_stages(a.cin, a.cout, cr, 32, 2))
      return cudaErrorInvalidValue;
    return res ? launch_dxn<32, 32, true, 2>(a, st, c.stages) : launch_dxn<32, 32, false, 2>(a, st, c.stages);
  }
  if (c.kind == 1) {
    if (!halo_ok(a.R, a.cout, a.cin, cr) || c.bn != a.cout || c.stages < 2 ||
        c.stages > halo_stages(a.cin, a.cout, cr, c.ck))
      return cudaErrorInvalidValue;
#define OMNI_HALO(BN_, CK_, RES_) \
    if (c.bn == BN_ && c.ck == CK_ && res == RES_) return launch_halo<BN_, CK_, RES_, 1>(a, st, c.stages);
    OMNI_HALO(32, 32, false) OMNI_HALO(32, 32, true) OMNI_HALO(32, 64, false) OMNI_HALO(32, 64, true)
    OMNI_HALO(64, 32, false) OMNI_HALO(64, 32, true) OMNI_HALO(64, 64, false) OMNI_HALO(64, 64, true)
#undef OMNI_HALO
    return cudaErrorInvalidValue;
  }
  if (c.kind == 3 || c.kind == 6) {
    if (!halo_ok(a.R, a.cout, a.cin, cr) || c.bn != a.cout || c.ck != 32 || c.stages < 2 ||
        c.stages > halo_stages(a.cin, a.cout, cr, 32, 2))
      return cudaErrorInvalidValue;
    if (c.kind == 6) {
      if (c.bn == 32) return res ? launch_halo<32, 32, true, 2, true>(a, st, c.stages) : launch_halo<32, 32, false, 2, true>(a, st, c.stages);
      if (c.bn == 64) return res ? launch_halo<64, 32, true, 2, true>(a, st, c.stages) : launch_halo<64, 32, false, 2, true>(a, st, c.stages);
      return cudaErrorInvalidValue;
    }
    if (c.bn == 32) return res ? launch_halo<32, 32, true, 2>(a, st, c.stages) : launch_halo<32, 32, false, 2>(a, st, c.stages);
    if (c.bn == 64) return res ? launch_halo<64, 32, true, 2>(a, st, c.stages) : launch_halo<64, 32, false, 2>(a, st, c.stages);
    return cudaErrorInvalidValue;
  }
  if (!pertap_ok(a.R, a.cin, a.cout, cr, c.bn, c.ck)) return cudaErrorInvalidValue;
  if (c.kind == 8) {
    if (c.ck != 64) return cudaErrorInvalidValue;
    if (c.bn == 128) return res ? launch_t<128, 64, true, true>(a, st) : launch_t<128, 64, false, true>(a, st);
    if (c.bn == 256 && !res) return launch_t<256, 64, false, true>(a, st);
    return cudaErrorInvalidValue;
  }
#define OMNI_TC(BN_, CK_, RES_) \
  if (c.bn == BN_ && c.ck == CK_ && res == RES_) return launch_t<BN_, CK_, RES_>(a, st);
  OMNI_TC(32, 32, false) OMNI_TC(32, 32, true) OMNI_TC(32, 64, false) OMNI_TC(32, 64, true)
  OMNI_TC(64, 32, false) OMNI_TC(64, 32, true) OMNI_TC(64, 64, false) OMNI_TC(64, 64, true)
  OMNI_TC(128, 32, false) OMNI_TC(128, 32, true) OMNI_TC(128, 64, false) OMNI_TC(128, 64, true)
  OMNI_TC(256, 32, false) OMNI_TC(256, 64, false)
#undef OMNI_TC
  return cudaErrorInvalidValue;
}

#if OMNI_TC_F16
cudaError_t launch_conv_first_tc_f16(const ConvArgs& a, cudaStream_t st) {
#else
cudaError_t launch_conv_first_tc_bf16(const ConvArgs& a, cudaStream_t st) {
#endif
  if (a.R < 16 || a.R % 16 || a.y_cs % 8 || a.y_co % 8 || reinterpret_cast<uintptr_t>(a.y) % 16 ||
      reinterpret_cast<uintptr_t>(a.w.w_bf16) % 16 || !a.cv.ptr[0] || !a.tiles3)
    return cudaErrorInvalidValue;
  for (int k = 0; k < kMaxCanvases; ++k)
    if (a.cv.ptr[k] && (a.cv.rows[k] < 1 || reinterpret_cast<uintptr_t>(a.cv.ptr[k]) % 16 || a.cv.stride[k] % 16))
      return cudaErrorInvalidValue;
  if (a.cout == 32) return launch_first<32>(a, st);
  if (a.cout == 64) return launch_first<64>(a, st);
  return cudaErrorInvalidValue;
}

#if !OMNI_TC_F16
bool conv_first_tc_supported(int R, int cout, const CanvasTab& cv) {
  if (!(R >= 16 && R % 16 == 0 && (cout == 32 || cout == 64)) || !cv.ptr[0]) return false;
  for (int k = 0; k < kMaxCanvases; ++k)
    if (cv.ptr[k] && (reinterpret_cast<uintptr_t>(cv.ptr[k]) % 16 || cv.stride[k] % 16)) return false;
  return true;
}

cudaError_t launch_conv_first_tc(const ConvArgs& a, cudaStream_t st) {
  return a.f16 ? launch_conv_first_tc_f16(a, st) : launch_conv_first_tc_bf16(a, st);
}

cudaError_t launch_conv_tc_cfg(const ConvArgs& a, const TcConfig& c, cudaStream_t st) {
  return a.f16 ? launch_conv_tc_cfg_f16(a, c, st) : launch_conv_tc_cfg_bf16(a, c, st);
}

cudaError_t launch_conv_tc_e4m3(const ConvArgs& a, const TcConfig& c, cudaStream_t st) {
  // x and the weights hold E4M3 bytes; per-tap kernel, one CTA (kind 0) or CTA
  // pairs (kind 8), 128-channel chunks, no projection or fused outputs
  if (a.res_mode != RES_NONE || a.pool || a.head_theta || !a.y || c.ck != 128) return cudaErrorInvalidValue;
  if (!pertap_ok(a.R, a.cin, a.cout, 0, c.bn, 128) || (c.bn != 128 && c.bn != 256)) return cudaErrorInvalidValue;
  if ((a.x_co % 16) || (a.x_cs % 16) || (a.y_co % 8) || (a.y_cs % 8) ||
      (reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.y) |
       reinterpret_cast<uintptr_t>(a.w.w_bf16)) % 16)
    return cudaErrorInvalidValue;
  if (c.kind == 0)
    return c.bn == 128 ? launch_t<128, 128, false, false, true>(a, st) : launch_t<256, 128, false, false, true>(a, st);
  if (c.kind == 8 && (long long)a.R * a.R % (2 * kBM) == 0)
    return c.bn == 128 ? launch_t<128, 128, false, true, true>(a, st) : launch_t<256, 128, false, true, true>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_conv_tc(const ConvArgs& a, cudaStream_t st) {
  const int cr = a.res_mode == RES_TENSOR ? a.cr : 0;
  if (!conv_tc_supported(a.R, a.cin, a.cout, cr)) return cudaErrorInvalidValue;
  return launch_conv_tc_cfg(a, tc_default(a.R, a.cin, a.cout, cr), st);
}
#endif

}  // namespace omni
