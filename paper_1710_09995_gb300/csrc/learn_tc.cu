// learn_tc.cu -- the accelerator's implicit-GEMM 3D convolution on the 5th-generation tensor
// cores: tcgen05.mma (kind::f16, bf16 x bf16 -> f32) issued by one thread, operands in shared
// memory in the canonical no-swizzle K-major layout, the 128 x N accumulator in tensor memory,
// read back with tcgen05.ld for the epilogue.
//
// A tile is 128 consecutive cells along x (one y, z, batch); GEMM view M = 128 cells,
// N = output channels (16 or 32), K = 27 taps x CIP input channels, issued as 27 x CIP/16 MMAs
// of K = 16.  Persistent CTAs of 128 threads; shared memory holds all weights and two
// 130 x 3 x 3-cell input boxes, as 8 x 16-byte core matrices:
//   box    element (cell c, channel k) at ((k / 8) NBOX + c) 8 + k % 8
//   weight element (tap t, out o, in k) at ((t CIP/8 + k / 8) N + o) 8 + k % 8
// so for tap t the A matrix of the tile starts at box cell (dz 3 + dy) 130 + dx (rows = cells,
// 8 consecutive rows one 128-byte core matrix, SBO 128 B, LBO = NBOX x 16 B along K) and the B
// matrix at weight group t CIP/8 (SBO 128 B, LBO = N x 16 B).
#include "internal.cuh"
#include "learn.cuh"

namespace gbcfd {
namespace learn {

using bf16 = __nv_bfloat16;

constexpr int TC_M = 128, TC_BX = TC_M + 2, TC_NBOX = TC_BX * 3 * 3, TC_THREADS = 128;

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

// tile k of this CTA -> (x0, y, z, b)
__device__ __forceinline__ void tc_tile(long long tile, const ConvArgs& A, int& x0, int& y, int& z, int& b) {
  const int tx = (A.X + TC_M - 1) / TC_M;
  x0 = (int)(tile % tx) * TC_M;
  tile /= tx;
  y = (int)(tile % A.Y);
  tile /= A.Y;
  z = (int)(tile % A.Z);
  b = (int)(tile / A.Z);
}

// input box of a tile: cell (bx, by, bz) = volume cell (x0 + bx - 1, y + by - 1, z + bz - 1), zero
// outside in x and y, periodic (or zero) in z
template <int CIP>
__device__ __forceinline__ void tc_stage_box(const ConvArgs& A, long long tile, bf16* box, int tid) {
  int x0, y, z, b;
  tc_tile(tile, A, x0, y, z, b);
  for (int i = tid; i < TC_NBOX * (CIP / 8); i += TC_THREADS) {
    const int c = i / (CIP / 8), kg = i % (CIP / 8);
    const int bx = c % TC_BX, by = (c / TC_BX) % 3, bz = c / (3 * TC_BX);
    const int gx = x0 + bx - 1, gy = y + by - 1;
    int gz = z + bz - 1;
    bool ok = gx >= 0 && gx < A.X && gy >= 0 && gy < A.Y;
    if (A.zper) gz = (gz + A.Z) % A.Z;
    else ok = ok && gz >= 0 && gz < A.Z;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (ok) v = *reinterpret_cast<const uint4*>(A.in + ((((long long)b * A.Z + gz) * A.Y + gy) * A.X + gx) * CIP + kg * 8);
    *reinterpret_cast<uint4*>(box + ((size_t)kg * TC_NBOX + c) * 8) = v;
  }
}

// the 27 x CIP/16 MMAs of one tile into the accumulator at tmem (one thread)
template <int CIP, int N>
__device__ __forceinline__ void tc_issue(unsigned box0, unsigned w0, unsigned tmem, unsigned bar) {
  constexpr unsigned idesc = instr_desc(N);
  for (int t = 0; t < NTAP; ++t) {
    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
    const unsigned cell0 = (unsigned)((dz * 3 + dy) * TC_BX + dx);
#pragma unroll
    for (int kk = 0; kk < CIP / 16; ++kk) {
      const unsigned a = box0 + ((unsigned)(2 * kk) * TC_NBOX + cell0) * 16u;
      const unsigned bw = w0 + ((unsigned)(t * (CIP / 8) + 2 * kk) * N) * 16u;
      tc_mma(tmem, smem_desc(a, TC_NBOX * 16u, 128u), smem_desc(bw, N * 16u, 128u), idesc, (t | kk) != 0);
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

// persistent: CTA c takes tiles c, c + G, c + 2G, ...; the weights are staged once, the input box
// and the 128 x N accumulator are double-buffered so that staging tile k+1 and the epilogue of
// tile k overlap the tensor-core work
template <int CIP, int N, int COP, int MODE>
__global__ void __launch_bounds__(TC_THREADS) conv_tc_kernel(const ConvArgs A, const bf16* __restrict__ wtc,
                                                             int* __restrict__ flag, long long ntiles) {
  extern __shared__ __align__(128) unsigned char smem[];
  bf16* wsm = reinterpret_cast<bf16*>(smem);                         // 27 x CIP x N
  bf16* boxes = wsm + NTAP * CIP * N;                                // 2 x TC_NBOX x CIP
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(boxes + 2 * TC_NBOX * CIP);  // 2
  unsigned* tslot = reinterpret_cast<unsigned*>(bar + 2);
  int* sabort = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int COLS = 2 * (N < 32 ? 32 : N);  // two accumulators

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
    *sabort = 0;
  }
  for (int i = tid; i < NTAP * N * (CIP / 8); i += TC_THREADS) {  // global [27][N][CIP] -> core matrices
    const int t = i / (N * (CIP / 8)), r = i % (N * (CIP / 8)), o = r / (CIP / 8), kg = r % (CIP / 8);
    const uint4 v = *reinterpret_cast<const uint4*>(wtc + ((size_t)t * N + o) * CIP + kg * 8);
    *reinterpret_cast<uint4*>(wsm + (((size_t)t * (CIP / 8) + kg) * N + o) * 8) = v;
  }
  const long long first = blockIdx.x, stride = gridDim.x;
  if (first < ntiles) tc_stage_box<CIP>(A, first, boxes, tid);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem0 = *tslot, colw = (unsigned)(N < 32 ? 32 : N);
  const unsigned w0 = smem_u32(wsm), boxa = smem_u32(boxes), bara = smem_u32(bar);
  constexpr unsigned BOXB = TC_NBOX * CIP * 2;  // bytes per box
  unsigned phase = 0;    // parity of each barrier's next completion
  unsigned issued = 0;   // barriers with an MMA group not yet waited for (thread 0's view is exact)
  if (first < ntiles && tid == 0) {
    tc_issue<CIP, N>(boxa, w0, tmem0, bara);
    issued |= 1u;
  }
  int k = 0;
  for (long long tile = first; tile < ntiles; tile += stride, ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    const long long tnext = tile + stride;
    if (tnext < ntiles) tc_stage_box<CIP>(A, tnext, boxes + nxt * TC_NBOX * CIP, tid);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // box k+1 staged; every thread is done with the epilogue of tile k-1
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (*sabort) break;
    if (tnext < ntiles && tid == 0) {
      tc_issue<CIP, N>(boxa + nxt * BOXB, w0, tmem0 + nxt * colw, bara + 8u * nxt);
      issued |= 1u << nxt;
    }
    // warp-uniform outcome: tcgen05.ld below is a whole-warp instruction
    const bool ok = __all_sync(0xffffffffu, mbar_wait_limited(bara + 8u * cur, (phase >> cur) & 1u));
    if (!ok) {
      if (tid == 0) atomicOr(flag, FLAG_TIMEOUT);
      atomicOr(sabort, 1);
      continue;  // the next barrier makes every thread see the abort
    }
    phase ^= 1u << cur;
    issued &= ~(1u << cur);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
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
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  }
  // an MMA group still in flight after an abort: give it a bounded wait before freeing its columns
  if (tid == 0)
    for (int j = 0; j < 2; ++j)
      if (issued & (1u << j)) mbar_wait_limited(bara + 8u * j, (phase >> j) & 1u);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem0), "r"(COLS));
}

template <int CIP, int N, int COP, int MODE>
static cudaError_t conv_tc_go(const ConvArgs& a, const bf16* wtc, int* flag, cudaStream_t s) {
  const size_t bytes = (size_t)(NTAP * CIP * N + 2 * TC_NBOX * CIP) * sizeof(bf16) + 32;
  static unsigned long long done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!(dev < 64 && ((done >> dev) & 1ull))) {
    e = cudaFuncSetAttribute(conv_tc_kernel<CIP, N, COP, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
    if (e != cudaSuccess) return e;
    if (dev < 64) done |= 1ull << dev;
  }
  int nsm = 0, occ = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv_tc_kernel<CIP, N, COP, MODE>, TC_THREADS, bytes);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)((a.X + TC_M - 1) / TC_M) * a.Y * a.Z * a.B;
  long long grid = (long long)nsm * (occ > 0 ? occ : 1);
  if (grid > tiles) grid = tiles;
  conv_tc_kernel<CIP, N, COP, MODE><<<(unsigned)grid, TC_THREADS, bytes, s>>>(a, wtc, flag, tiles);
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
