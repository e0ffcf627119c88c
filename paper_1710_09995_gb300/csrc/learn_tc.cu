// learn_tc.cu -- the accelerator's implicit-GEMM 3D convolution on the 5th-generation tensor
// cores: tcgen05.mma (kind::f16, bf16 x bf16 -> f32) issued by one thread, operands in shared
// memory in the canonical no-swizzle K-major layout, the 128 x N accumulator in tensor memory,
// read back with tcgen05.ld for the epilogue.
//
// A tile is 128 consecutive cells along x (one y, z, batch); GEMM view M = 128 cells,
// N = output channels (16 or 32), K = 27 taps x CIP input channels, issued as 27 x CIP/16 MMAs
// of K = 16.  Persistent CTAs of 128 threads; shared memory holds all weights and two input
// boxes of 3 x 3 rows of 130 cells (rows padded to 136), as 8 x 16-byte core matrices:
//   box    element (row r, cell c, channel k) at ((k / 8) NBOX + 136 r + c) 8 + k % 8
//   weight element (tap t, out o, in k) at ((t CIP/8 + k / 8) N + o) 8 + k % 8
// so for tap t the A matrix of the tile starts at box cell (dz 3 + dy) 136 + dx (rows = cells,
// 8 consecutive rows one 128-byte core matrix, SBO 128 B, LBO = NBOX x 16 B along K) and the B
// matrix at weight group t CIP/8 (SBO 128 B, LBO = N x 16 B).  The boxes are filled by TMA.
#include <atomic>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "learn.cuh"

namespace gbcfd {
namespace learn {

using bf16 = __nv_bfloat16;

constexpr int TC_M = 128, TC_BX = TC_M + 2, TC_RP = 136, TC_NBOX = TC_RP * 3 * 3, TC_THREADS = 128;
// a box row (130 cells) is padded to TC_RP = 136 cells so that every row of every channel group
// starts on a 128-byte boundary (the TMA destination alignment)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets, no swizzle
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version for this architecture; base offset 0, layout: no swizzle
  return d;
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, N, M = 128
__host__ __device__ constexpr unsigned instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned tmem, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait_limited(unsigned bar, unsigned parity) {
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > 2000000000ull) return false;  // 2 s
  }
}

// tile -> (x0, y, z, b)
__device__ __forceinline__ void tc_tile(long long tile, const ConvArgs& A, int& x0, int& y, int& z, int& b) {
  const int tx = (A.X + TC_M - 1) / TC_M;
  x0 = (int)(tile % tx) * TC_M;
  tile /= tx;
  y = (int)(tile % A.Y);
  tile /= A.Y;
  z = (int)(tile % A.Z);
  b = (int)(tile / A.Z);
}

// the input box of a tile by TMA: for each of the 3 x 3 (y, z) rows and each 8-channel group one
// 130 x 16-byte copy of the activation tensor viewed as [Z B][Y][X][CIP/8][8], box (8, 1, 130,
// 1, 1) at x0 - 1; the copy unit fills x and y outside the volume with zeros.  Rows outside the
// volume in a non-periodic z are zeroed by the threads (a z - 1 row would otherwise belong to
// the previous batch).  Thread 0 issues the copies; returns the bytes the barrier expects.
template <int CIP>
__device__ __forceinline__ void tc_load_box(const ConvArgs& A, const CUtensorMap* map, long long tile, unsigned box,
                                            unsigned bar, int tid) {
  int x0, y, z, b;
  tc_tile(tile, A, x0, y, z, b);
  if (tid == 0) {
    unsigned bytes = 0;
    for (int r = 0; r < 9; ++r) {
      int zz = z + r / 3 - 1;
      if (A.zper) zz = (zz + A.Z) % A.Z;
      if (zz >= 0 && zz < A.Z) bytes += (CIP / 8) * TC_BX * 16u;
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
    for (int r = 0; r < 9; ++r) {
      const int by = r % 3, bz = r / 3;
      int zz = z + bz - 1;
      if (A.zper) zz = (zz + A.Z) % A.Z;
      if (zz < 0 || zz >= A.Z) continue;
      for (int kg = 0; kg < CIP / 8; ++kg) {
        const unsigned dst = box + (unsigned)((kg * TC_NBOX + r * TC_RP) * 16);
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
            "%6}], [%7];\n" ::"r"(dst),
            "l"(reinterpret_cast<unsigned long long>(map)), "r"(0), "r"(kg), "r"(x0 - 1), "r"(y + by - 1),
            "r"(b * A.Z + zz), "r"(bar)
            : "memory");
      }
    }
  }
  if (!A.zper) {  // zero rows outside the volume in z
    for (int r = 0; r < 9; r += 3) {
      const int zz = z + r / 3 - 1;
      if (zz >= 0 && zz < A.Z) continue;
      for (int i = tid; i < 3 * (CIP / 8) * TC_RP; i += TC_THREADS) {
        const int kg = i / (3 * TC_RP), rest = i % (3 * TC_RP);
        bf16* p = reinterpret_cast<bf16*>(__cvta_shared_to_generic(box)) + ((size_t)kg * TC_NBOX + r * TC_RP + rest) * 8;
        *reinterpret_cast<uint4*>(p) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }
}

// the 27 x CIP/16 MMAs of one tile into the accumulator at tmem (one thread), then a commit
template <int CIP, int N>
__device__ __forceinline__ void tc_issue(unsigned box0, unsigned w0, unsigned tmem, unsigned bar) {
  constexpr unsigned idesc = instr_desc(N);
  for (int t = 0; t < NTAP; ++t) {
    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
    const unsigned cell0 = (unsigned)((dz * 3 + dy) * TC_RP + dx);
#pragma unroll
    for (int kk = 0; kk < CIP / 16; ++kk) {
      const unsigned a = box0 + ((unsigned)(2 * kk) * TC_NBOX + cell0) * 16u;
      const unsigned bw = w0 + ((unsigned)(t * (CIP / 8) + 2 * kk) * N) * 16u;
      tc_mma(tmem, smem_desc(a, TC_NBOX * 16u, 128u), smem_desc(bw, N * 16u, 128u), idesc, (t | kk) != 0);
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

// persistent: CTA c takes tiles c, c + G, c + 2G, ...; the weights are staged once; two input
// boxes (loaded by TMA) and two tensor-memory accumulators let the copies of tile k+2 and the
// MMAs of tile k+1 run during the epilogue of tile k
template <int CIP, int N, int COP, int MODE>
__global__ void __launch_bounds__(TC_THREADS) conv_tc_kernel(const ConvArgs A, const __grid_constant__ CUtensorMap map,
                                                             const bf16* __restrict__ wtc, int* __restrict__ flag,
                                                             long long ntiles) {
  extern __shared__ __align__(128) unsigned char smem[];
  bf16* boxes = reinterpret_cast<bf16*>(smem);                      // 2 x TC_NBOX x CIP (128-byte rows)
  bf16* wsm = boxes + 2 * TC_NBOX * CIP;                            // 27 x CIP x N
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(wsm + NTAP * CIP * N);  // full[2], done[2]
  unsigned* tslot = reinterpret_cast<unsigned*>(bar + 4);
  int* sabort = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int COLS = 2 * (N < 32 ? 32 : N);
  constexpr unsigned BOXB = TC_NBOX * CIP * 2;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int j = 0; j < 4; ++j) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar + j)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
    *sabort = 0;
  }
  for (int i = tid; i < NTAP * N * (CIP / 8); i += TC_THREADS) {  // global [27][N][CIP] -> core matrices
    const int t = i / (N * (CIP / 8)), r = i % (N * (CIP / 8)), o = r / (CIP / 8), kg = r % (CIP / 8);
    const uint4 v = *reinterpret_cast<const uint4*>(wtc + ((size_t)t * N + o) * CIP + kg * 8);
    *reinterpret_cast<uint4*>(wsm + (((size_t)t * (CIP / 8) + kg) * N + o) * 8) = v;
  }
  __syncthreads();  // barriers initialised
  const unsigned boxa = smem_u32(boxes), w0 = smem_u32(wsm), full0 = smem_u32(bar), done0 = smem_u32(bar + 2);
  const long long first = blockIdx.x, stride = gridDim.x;
  tc_load_box<CIP>(A, &map, first, boxa, full0, tid);
  if (first + stride < ntiles) tc_load_box<CIP>(A, &map, first + stride, boxa + BOXB, full0 + 8u, tid);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem0 = *tslot, colw = (unsigned)(N < 32 ? 32 : N);
  unsigned fphase = 0, dphase = 0;  // parities of the next completion of full[j] / done[j]
  unsigned inflight = 0;            // thread 0: copy groups (bits 0-1) and MMA groups (bits 2-3) not yet waited for
  if (tid == 0) {
    inflight = (first + stride < ntiles) ? 3u : 1u;
    const bool ok = mbar_wait_limited(full0, 0u);
    fphase ^= 1u;
    inflight &= ~1u;
    if (ok) {
      tc_issue<CIP, N>(boxa, w0, tmem0, done0);
      inflight |= 4u;
    } else {
      atomicOr(flag, FLAG_TIMEOUT);
      *sabort = 1;
    }
  }
  __syncthreads();
  int k = 0;
  for (long long tile = first; tile < ntiles && !*sabort; tile += stride, ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    // MMA(k) done: box[cur] and tensor memory [cur] hold tile k's results
    const bool ok = __all_sync(0xffffffffu, mbar_wait_limited(done0 + 8u * cur, (dphase >> cur) & 1u));
    if (!ok) {
      if (tid == 0) atomicOr(flag, FLAG_TIMEOUT);
      atomicOr(sabort, 1);
      __syncthreads();
      break;
    }
    dphase ^= 1u << cur;
    if (tid == 0) inflight &= ~(4u << cur);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tile + 2 * stride < ntiles) {  // copies of tile k+2 into the box tile k used
      tc_load_box<CIP>(A, &map, tile + 2 * stride, boxa + cur * BOXB, full0 + 8u * cur, tid);
      if (tid == 0) inflight |= 1u << cur;
    }
    if (tid == 0 && tile + stride < ntiles) {  // MMA(k+1) once its box has landed
      const bool okf = mbar_wait_limited(full0 + 8u * nxt, (fphase >> nxt) & 1u);
      fphase ^= 1u << nxt;
      inflight &= ~(1u << nxt);
      if (okf) {
        tc_issue<CIP, N>(boxa + nxt * BOXB, w0, tmem0 + nxt * colw, done0 + 8u * nxt);
        inflight |= 4u << nxt;
      } else {
        atomicOr(flag, FLAG_TIMEOUT);
        *sabort = 1;
      }
    }
    int x0, y, z, b;
    tc_tile(tile, A, x0, y, z, b);
    float acc[32];
    const unsigned taddr = tmem0 + cur * colw + ((unsigned)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=f"(acc[0]), "=f"(acc[1]), "=f"(acc[2]), "=f"(acc[3]), "=f"(acc[4]), "=f"(acc[5]), "=f"(acc[6]),
          "=f"(acc[7]), "=f"(acc[8]), "=f"(acc[9]), "=f"(acc[10]), "=f"(acc[11]), "=f"(acc[12]), "=f"(acc[13]),
          "=f"(acc[14]), "=f"(acc[15]), "=f"(acc[16]), "=f"(acc[17]), "=f"(acc[18]), "=f"(acc[19]),
          "=f"(acc[20]), "=f"(acc[21]), "=f"(acc[22]), "=f"(acc[23]), "=f"(acc[24]), "=f"(acc[25]),
          "=f"(acc[26]), "=f"(acc[27]), "=f"(acc[28]), "=f"(acc[29]), "=f"(acc[30]), "=f"(acc[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    const int gx = x0 + tid;
    if (gx < A.X) {
      const long long cell = (((long long)b * A.Z + z) * A.Y + y) * A.X + gx;
      if constexpr (MODE == FWD_SILU) {
        __align__(16) bf16 o[COP];
#pragma unroll
        for (int c = 0; c < COP; ++c) {
          const float v = acc[c] + A.bias[c];
          if (A.zsave) A.zsave[cell * COP + c] = v;
          o[c] = __float2bfloat16(v / (1.0f + __expf(-v)));
        }
#pragma unroll
        for (int q = 0; q < COP / 8; ++q)
          reinterpret_cast<uint4*>(static_cast<bf16*>(A.out) + cell * COP)[q] = reinterpret_cast<const uint4*>(o)[q];
      } else if constexpr (MODE == FWD_LINEAR) {
        float* out = static_cast<float*>(A.out) + cell * COP;
#pragma unroll
        for (int c = 0; c < COP; ++c) out[c] = acc[c] + A.bias[c];
      } else {
        __align__(16) bf16 o[COP];
#pragma unroll
        for (int c = 0; c < COP; ++c) {
          const float zp = A.zprev[cell * COP + c];
          const float sg = 1.0f / (1.0f + __expf(-zp));
          o[c] = __float2bfloat16(acc[c] * (sg * (1.0f + zp * (1.0f - sg))));
        }
#pragma unroll
        for (int q = 0; q < COP / 8; ++q)
          reinterpret_cast<uint4*>(static_cast<bf16*>(A.out) + cell * COP)[q] = reinterpret_cast<const uint4*>(o)[q];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // zeroed rows of box[cur]
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // tensor memory [cur] read by everyone; zero rows written
  }
  // after an abort: give copies and MMAs still in flight a bounded wait before freeing anything
  if (tid == 0)
    for (int j = 0; j < 2; ++j) {
      if (inflight & (1u << j)) mbar_wait_limited(full0 + 8u * j, (fphase >> j) & 1u);
      if (inflight & (4u << j)) mbar_wait_limited(done0 + 8u * j, (dphase >> j) & 1u);
    }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem0), "r"(COLS));
}

// the TMA map of an activation tensor [Z B][Y][X][CIP] as 5 dimensions (8, CIP/8, X, Y, Z B)
static cudaError_t tc_map(CUtensorMap* m, const void* base, int CIP, const ConvArgs& a) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return cudaErrorNotSupported;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  cuuint64_t dims[5] = {8, (cuuint64_t)(CIP / 8), (cuuint64_t)a.X, (cuuint64_t)a.Y, (cuuint64_t)a.Z * a.B};
  cuuint64_t strides[4] = {16, (cuuint64_t)CIP * 2, (cuuint64_t)a.X * CIP * 2, (cuuint64_t)a.Y * a.X * CIP * 2};
  cuuint32_t box[5] = {8, 1, (cuuint32_t)TC_BX, 1, 1};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CIP, int N, int COP, int MODE>
static cudaError_t conv_tc_go(const ConvArgs& a, const bf16* wtc, int* flag, cudaStream_t s) {
  const size_t bytes = (size_t)(2 * TC_NBOX * CIP + NTAP * CIP * N) * sizeof(bf16) + 64;
  static std::atomic<unsigned long long> done{0};  // per-device bit; host threads may race here
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!(dev < 64 && ((done.load(std::memory_order_acquire) >> dev) & 1ull))) {
    e = cudaFuncSetAttribute(conv_tc_kernel<CIP, N, COP, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
    if (e != cudaSuccess) return e;
    if (dev < 64) done.fetch_or(1ull << dev, std::memory_order_acq_rel);
  }
  if (((uintptr_t)a.in & 15u) != 0) return cudaErrorMisalignedAddress;
  CUtensorMap map;
  e = tc_map(&map, a.in, CIP, a);
  if (e != cudaSuccess) return e;
  int nsm = 0, occ = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv_tc_kernel<CIP, N, COP, MODE>, TC_THREADS, bytes);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((a.X + TC_M - 1) / TC_M) * a.Y * a.Z * a.B;
  long long grid = (long long)nsm * (occ > 0 ? occ : 1);
  if (grid > tiles) grid = tiles;
  conv_tc_kernel<CIP, N, COP, MODE><<<(unsigned)grid, TC_THREADS, bytes, s>>>(a, map, wtc, flag, tiles);
  return cudaGetLastError();
}

// layers 1..3 forward; layers 3 and 2 backward-data (taps mirrored, channels swapped, x SiLU')
cudaError_t launch_conv(int layer, int mode, const ConvArgs& a, int* flag, cudaStream_t s) {
  if (mode == FWD_SILU && layer == 1) return conv_tc_go<P0, P1, P1, FWD_SILU>(a, a.w, flag, s);
  if (mode == FWD_SILU && layer == 2) return conv_tc_go<P1, P2, P2, FWD_SILU>(a, a.w, flag, s);
  if (mode == FWD_LINEAR && layer == 3) return conv_tc_go<P2, 16, P3, FWD_LINEAR>(a, a.w, flag, s);
  if (mode == BWD_DSILU && layer == 3) return conv_tc_go<16, P2, P2, BWD_DSILU>(a, a.w, flag, s);  // dY -> dZ2
  if (mode == BWD_DSILU && layer == 2) return conv_tc_go<P2, P1, P1, BWD_DSILU>(a, a.w, flag, s);  // dZ2 -> dZ1
  return cudaErrorInvalidValue;
}

}  // namespace learn
}  // namespace gbcfd
