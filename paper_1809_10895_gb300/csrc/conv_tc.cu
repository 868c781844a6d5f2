// conv_tc.cu -- the 32 -> 32 channel 3x3x3 convolution of the warm-start
// network on the 5th-generation tensor cores: tcgen05.mma with operands in
// shared memory (staged by TMA) and FP32 accumulators in tensor memory.
//
// Implicit GEMM over a tile of 32 x 6 x 2 output voxels (x, y, z).  The input
// tile with its one-voxel halo (34 x 8 x 4 voxels) is copied by four bulk
// tensor copies, one per group of 8 channels; each copy lands as a "plane" of
// 16-byte rows in halo-linear voxel order hl = (z (H+2) + y) (W+2) + x, which
// is the K-major, no-swizzle operand layout (core matrices of 8 rows x 16
// bytes).  For a filter tap (dz, dy, dx) the A operand of GEMM rows hl is the
// same plane read from hl + off(tap), off = (dz (Ty+2) + dy) (Tx+2) + dx, so
// every tap is a shifted descriptor of the same shared-memory tile.  Output
// rows hl run over the tile's interior span in four blocks of M = 128;
// rows on the halo ring are computed and discarded.  N = 32 output channels,
// K = 16 per instruction (two 8-channel planes), 27 taps x 2 = 54 MMAs per
// row block.  The weights (32 x 864) sit in shared memory for the whole
// kernel in the same layout.
//
// Warp roles (persistent, one CTA per SM): warp 5 lane 0 issues the tensor
// copies (two input stages), warp 4 lane 0 the MMAs (two accumulator stages
// of 4 x 32 TMEM columns), warps 0-3 the epilogue (tcgen05.ld of one TMEM lane
// = one voxel's 32 channels per thread; bias, residual, ReLU; BF16 / FP32
// stores).  Every mbarrier wait is bounded: a wait that runs out raises the
// CTA's abort flag and the device fault flag, every role leaves its loop,
// and TMEM is freed before the kernel returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nn.cuh"
#include "tma.cuh"

namespace rf {
namespace nn {

namespace {

constexpr int TC_TX = 32, TC_TY = 6, TC_TZ = 2;                      // output tile
constexpr int TC_HX = TC_TX + 2, TC_HY = TC_TY + 2, TC_HZ = TC_TZ + 2;   // halo box
constexpr int TC_HALO = TC_HX * TC_HY * TC_HZ;                           // 1088 voxels
constexpr int TC_ROW0 = (TC_HY + 1) * TC_HX + 1;                         // first interior hl (307)
constexpr int TC_OFFMAX = TC_HY * TC_HX + TC_HX + 1;                     // largest |tap offset| (307)
constexpr int TC_RB = 4;                                                 // row blocks of 128
constexpr int TC_PLANE_ROWS = 1152;   // >= TC_ROW0 + 128 TC_RB + TC_OFFMAX - 1 (rows past 1088 feed discarded outputs)
constexpr int TC_PLANE_BYTES = TC_PLANE_ROWS * 16;                       // 18 432
constexpr int TC_BOX_BYTES = TC_HALO * 16;                               // 17 408 per plane copy
constexpr int TC_THREADS = 192;
constexpr int TC_WAIT_TRIES = 1 << 20;

// Per instantiation: CINP input channels (16 or 32, in planes of 8), NOUT
// GEMM columns (16 or 32).
template <int CINP, int NOUT>
struct TcShape {
    static constexpr int PLANES = CINP / 8;
    static constexpr int KC = CINP / 16;                      // K = 16 chunks per tap
    static constexpr int KP = 27 * CINP;                      // weights per output channel
    static constexpr int A_BYTES = PLANES * TC_PLANE_BYTES;   // per stage
    static constexpr int B_BYTES = (KP / 8) * NOUT * 16;
    static constexpr int SMEM = 2 * A_BYTES + B_BYTES + 1024;
    static constexpr int TMEM_COLS = 2 * 4 * NOUT;            // 2 stages x 4 row blocks
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NOUT >> 3) << 17) |
                                      ((128u >> 4) << 24);
    static_assert(CINP == 16 || CINP == 32, "input planes");
    static_assert(NOUT == 16 || NOUT == 32, "M = 128 needs N a multiple of 16");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

static_assert(TC_ROW0 + 128 * TC_RB - 1 + TC_OFFMAX < TC_PLANE_ROWS, "plane rows cover every shifted read");
static_assert(TC_ROW0 + 128 * TC_RB - 1 >= (TC_TZ * TC_HY + TC_TY) * TC_HX + TC_TX, "row blocks cover the interior");
static_assert(TC_PLANE_BYTES % 1024 == 0, "TMA destinations 128-byte aligned, stages 1024-byte aligned");

struct TcParams {
    int B, D, H, W;
    int ntx, nty, ntz;       // tiles along x, y, z
    long long tiles;
};

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    // K-major, no swizzle: start, leading (K-direction core-matrix) and stride
    // (8-row group) byte offsets >> 4, descriptor version 1 at bit 46
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// kind::f16 MMA, M = 128: D FP32, A and B BF16, both K-major (idesc).
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// 16 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Bounded wait that also gives up when another role raised the abort flag.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    for (int t = 0; t < TC_WAIT_TRIES; t++) {
        if (mbar_try_wait_sleep(bar, parity, 1000u)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void tile_origin(const TcParams &p, long long tile, int &b, int &z0, int &y0, int &x0)
{
    long long r = tile;
    const int tx = (int)(r % p.ntx);
    r /= p.ntx;
    const int ty = (int)(r % p.nty);
    r /= p.nty;
    const int tz = (int)(r % p.ntz);
    b = (int)(r / p.ntz);
    x0 = tx * TC_TX;
    y0 = ty * TC_TY;
    z0 = tz * TC_TZ;
}

}  // namespace

// Wb: NOUT x 27 CINP BF16 weights, K = tap CINP + c.  The input tensor has
// cin_mem channels (8 or 32); planes past cin_mem / 8 stay zero.  out_ch
// output channels (<= NOUT) are written, the row stride of out_b / out_f.
template <int CINP, int NOUT>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_conv3d_tc(TcParams p, const __grid_constant__ CUtensorMap in_map, int cin_mem, int out_ch,
            const __nv_bfloat16 *__restrict__ Wb, const float *__restrict__ bias,
            const __nv_bfloat16 *__restrict__ res, __nv_bfloat16 *__restrict__ out_b, float *__restrict__ out_f,
            int relu, int *fault)
{
    using S = TcShape<CINP, NOUT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = smem;                       // 2 stages x PLANES planes
    unsigned char *sB = smem + 2 * S::A_BYTES;      // weights, [k/8][n][8 k]
    const int loaded = cin_mem / 8;                 // planes filled by tensor copies
    __shared__ __align__(8) uint64_t full_bar[2], free_bar[2], tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    // tiles whose copies were issued / consumed, whose MMAs were committed /
    // drained by the epilogue (for the drain after an abort)
    __shared__ int s_issued, s_consumed, s_committed, s_drained;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    // weights into shared memory, zero planes for the channels the input does
    // not have (generic stores, then made visible to the async proxy)
    for (int e = threadIdx.x; e < (S::KP / 8) * NOUT; e += TC_THREADS) {
        const int n = e % NOUT, kg = e / NOUT;
        const uint4 w = *reinterpret_cast<const uint4 *>(Wb + (size_t)n * S::KP + kg * 8);
        *reinterpret_cast<uint4 *>(sB + (size_t)(kg * NOUT + n) * 16) = w;
    }
    for (int st = 0; st < 2; st++)
        for (int pl = loaded; pl < S::PLANES; pl++) {
            uint4 *z = reinterpret_cast<uint4 *>(sA + st * S::A_BYTES + pl * TC_PLANE_BYTES);
            for (int e = threadIdx.x; e < TC_PLANE_ROWS; e += TC_THREADS) z[e] = make_uint4(0u, 0u, 0u, 0u);
        }
    fence_proxy_async_smem();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++) {
            mbar_init(&full_bar[i], 1);
            mbar_init(&free_bar[i], 1);
            mbar_init(&tfull_bar[i], 1);
            mbar_init(&tempty_bar[i], 128);
        }
        mbar_init_fence();
        s_abort = 0;
        s_issued = s_consumed = s_committed = s_drained = 0;
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *abort_flag = &s_abort;

    if (warp == 5) {
        // ---------------- producer: halo tiles by tensor copies
        if (lane == 0) {
            int i = 0;
            for (long long tile = blockIdx.x; tile < p.tiles; tile += gridDim.x, i++) {
                const int s = i & 1;
                if (i >= 2 && !wait_or_abort(&free_bar[s], ((i >> 1) - 1) & 1, abort_flag)) break;
                int b, z0, y0, x0;
                tile_origin(p, tile, b, z0, y0, x0);
                mbar_expect_tx(&full_bar[s], loaded * TC_BOX_BYTES);
                unsigned char *dst = sA + s * S::A_BYTES;
                for (int cg = 0; cg < loaded; cg++) {
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];"
                        ::"r"(smem_addr(dst + cg * TC_PLANE_BYTES)), "l"(reinterpret_cast<uint64_t>(&in_map)),
                          "r"(smem_addr(&full_bar[s])), "r"(cg * 8), "r"(x0 - 1), "r"(y0 - 1), "r"(z0 - 1), "r"(b)
                        : "memory");
                }
                s_issued = i + 1;
            }
        }
    } else if (warp == 4) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int i = 0;
            for (long long tile = blockIdx.x; tile < p.tiles; tile += gridDim.x, i++) {
                const int s = i & 1;
                if (!wait_or_abort(&full_bar[s], (i >> 1) & 1, abort_flag)) break;
                s_consumed = i + 1;
                if (i >= 2 && !wait_or_abort(&tempty_bar[s], ((i >> 1) - 1) & 1, abort_flag)) break;
                tc_fence_after();
                const uint32_t a_base = smem_addr(sA + s * S::A_BYTES);
                const uint32_t b_base = smem_addr(sB);
                for (int rb = 0; rb < TC_RB; rb++) {
                    const uint32_t d = tmem + (uint32_t)((s * 4 + rb) * NOUT);
                    const int r0 = TC_ROW0 + 128 * rb;
                    for (int tap = 0; tap < 27; tap++) {
                        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                        const int off = (dz * TC_HY + dy) * TC_HX + dx;
                        for (int kc = 0; kc < S::KC; kc++) {
                            // A: planes 2kc, 2kc+1 (LBO) from row r0 + off; B: k-groups tap CINP/8 + 2kc, + 1
                            const uint64_t ad =
                                smem_desc(a_base + (uint32_t)(2 * kc * TC_PLANE_BYTES + (r0 + off) * 16), TC_PLANE_BYTES, 128);
                            const uint64_t bd = smem_desc(
                                b_base + (uint32_t)((tap * S::PLANES + 2 * kc) * NOUT * 16), NOUT * 16, 128);
                            tc_mma(d, ad, bd, S::IDESC, (tap | kc) ? 1u : 0u);
                        }
                    }
                }
                tc_commit(&free_bar[s]);
                tc_commit(&tfull_bar[s]);
                s_committed = i + 1;
            }
        }
    } else {
        // ---------------- epilogue: warps 0-3, TMEM lanes 32 warp .. 32 warp + 31
        int i = 0;
        const long long HW = (long long)p.H * p.W;
        for (long long tile = blockIdx.x; tile < p.tiles; tile += gridDim.x, i++) {
            const int s = i & 1;
            if (!wait_or_abort(&tfull_bar[s], (i >> 1) & 1, abort_flag)) break;
            if (threadIdx.x == 0) s_drained = i + 1;
            tc_fence_after();
            int b, z0, y0, x0;
            tile_origin(p, tile, b, z0, y0, x0);
            for (int rb = 0; rb < TC_RB; rb++) {
                float v[32];
                __syncwarp();
                const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((s * 4 + rb) * NOUT);
                if constexpr (NOUT == 32) {
                    tc_ld32(taddr, v);
                } else {
                    float v16[16];
                    tc_ld16(taddr, v16);
#pragma unroll
                    for (int c = 0; c < 16; c++) v[c] = v16[c];
                }
                const int hl = TC_ROW0 + 128 * rb + 32 * warp + lane;
                const int hx = hl % TC_HX, hy = (hl / TC_HX) % TC_HY, hz = hl / (TC_HX * TC_HY);
                const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
                const bool interior = hx >= 1 && hx <= TC_TX && hy >= 1 && hy <= TC_TY && hz >= 1 && hz <= TC_TZ;
                if (!interior || x >= p.W || y >= p.H || z >= p.D) continue;
                const long long m = x + (long long)p.W * y + HW * (z + (long long)p.D * b);
                if (out_ch == 32) {
#pragma unroll
                    for (int c = 0; c < 32; c++) v[c] += bias ? __ldg(&bias[c]) : 0.0f;
                    if (res) {
                        const uint4 *r4 = reinterpret_cast<const uint4 *>(res + m * 32);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const uint4 u = __ldg(&r4[q]);
                            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                            for (int h = 0; h < 4; h++) {
                                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[h]));
                                v[8 * q + 2 * h] += f.x;
                                v[8 * q + 2 * h + 1] += f.y;
                            }
                        }
                    }
                    if (relu) {
#pragma unroll
                        for (int c = 0; c < 32; c++) v[c] = fmaxf(v[c], 0.0f);
                    }
                    if (out_b) {
                        uint4 *o4 = reinterpret_cast<uint4 *>(out_b + m * 32);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            uint32_t w[4];
#pragma unroll
                            for (int h = 0; h < 4; h++) {
                                const __nv_bfloat162 t = __floats2bfloat162_rn(v[8 * q + 2 * h], v[8 * q + 2 * h + 1]);
                                w[h] = *reinterpret_cast<const uint32_t *>(&t);
                            }
                            o4[q] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                    if (out_f) {
                        float4 *o4 = reinterpret_cast<float4 *>(out_f + m * 32);
#pragma unroll
                        for (int q = 0; q < 8; q++)
                            o4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                } else {
                    // 8 output channels (the output convolution): FP32 out only
#pragma unroll
                    for (int c = 0; c < 8; c++) v[c] += bias ? __ldg(&bias[c]) : 0.0f;
                    if (relu) {
#pragma unroll
                        for (int c = 0; c < 8; c++) v[c] = fmaxf(v[c], 0.0f);
                    }
                    if (out_f) {
                        float4 *o4 = reinterpret_cast<float4 *>(out_f + m * 8);
                        o4[0] = make_float4(v[0], v[1], v[2], v[3]);
                        o4[1] = make_float4(v[4], v[5], v[6], v[7]);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty_bar[s]);
        }
    }

    // every role is done (or aborted): wait out this CTA's copies and MMAs,
    // then free the tensor memory
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) {
        atomicExch(fault, 1);
        // copies issued but not consumed, MMAs committed but not drained
        for (int j = s_consumed; j < s_issued; j++) mbar_wait_bounded(&full_bar[j & 1], (j >> 1) & 1, TC_WAIT_TRIES);
        for (int j = s_drained; j < s_committed; j++) mbar_wait_bounded(&tfull_bar[j & 1], (j >> 1) & 1, TC_WAIT_TRIES);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    __syncwarp();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS) : "memory");
}

// ------------------------------------------------------------ weight gradient
// Weight and bias gradient of a 32 -> 32 convolution on the tcgen05 tensor
// cores:
//   dW[co][tap 32 + ci] += sum_v X[v + off(tap)][ci] G[v][co],   db[co] += sum_v G[v][co].
// GEMM: M = (dy, ci), N = co, K = voxels.  The contraction runs over the
// voxels, the outer index of both channels-last operands, so both are
// transposed into K-major tiles in shared memory.  Per tile of 32 x 4 x 2
// output voxels:
//   X's halo tile (34 x 6 x 4 voxels) lands by four bulk tensor copies (one
//     per 8-channel plane, 16-byte rows in halo-linear order), and is
//     transposed by ldmatrix.trans into three copies
//     T_dx[(z', y', ci)][x] = X[x + dx][y'][z'][ci], dx = -1, 0, 1, over the
//     tile's halo rows (z', y') and its 32 x positions;
//   G_T[(z, y)][co][x] = G[x][y][z][co] over the interior rows (zero outside
//     the volume), from 4-byte pairs loaded a tile ahead and transposed by
//     movmatrix.
// For tap (dz, dy, dx) and output row (y, z) the A operand is T_dx at row
// (z + dz, y + dy); the three dy taps are consecutive blocks of 32 rows, so
// one M = 128 MMA covers dy = -1, 0, 1 (its fourth block of 32 rows is
// discarded).  Per output row: 9 (dz, dx) chains of K = 32 (two MMAs of
// K = 16) into 9 accumulators of 32 TMEM columns, which hold the CTA's sums
// over all its tiles; then one atomic add per weight per CTA.  The bias
// gradient is summed from the G pairs as they arrive.  The next tile's copy
// is issued as soon as the current one is transposed, so it flies while the
// MMAs run; the transposed operands are single-buffered (every thread waits,
// bounded, for the MMAs before they are rewritten).
constexpr int WT_TX = 32, WT_TY = 4, WT_TZ = 2;
constexpr int WT_HX = WT_TX + 2, WT_HY = WT_TY + 2, WT_HZ = WT_TZ + 2;
constexpr int WT_ROWS = (WT_HZ * WT_HY + 1) * 32;   // (z', y', ci) rows, plus one block of 32 read into discarded rows
constexpr int WT_LBO = WT_ROWS * 16;                // bytes between the K groups (8 x positions) of a copy
constexpr int WT_COPY = 4 * WT_LBO;                 // one dx copy: 32 x positions
constexpr int WT_GROW = 4 * 32 * 16;                // one interior row of G_T: 4 K groups x 32 co x 16 bytes
constexpr int WT_XPLANE = WT_HX * WT_HY * WT_HZ * 16;   // one 8-channel plane of the halo tile
constexpr int WT_OFF_G = 3 * WT_COPY, WT_OFF_X = WT_OFF_G + WT_TY * WT_TZ * WT_GROW;
constexpr int WT_SMEM = WT_OFF_X + 4 * WT_XPLANE + 1024;
constexpr int WT_THREADS = 256, WT_WARPS = WT_THREADS / 32;
constexpr int WT_XQUADS = 3 * WT_HZ * WT_HY * 4;    // ldmatrix.x4 of the three copies (4 K groups each)
constexpr int WT_TMEM_COLS = 512;                   // 9 x 32 used
constexpr int WT_KP = 27 * 32;                      // weights per output channel
static_assert(WT_XQUADS % WT_WARPS == 0, "whole rounds of transposes");
static_assert(WT_TY * WT_TZ * 4 * 2 == 2 * 32, "G_T blocks: 16 per warp, the warp's channel block fixed");
static_assert(WT_SMEM <= 227 * 1024, "shared memory");
static_assert(WT_LBO / 16 < (1 << 14), "descriptor offset field");
static_assert(WT_XPLANE % 128 == 0 && WT_OFF_X % 128 == 0, "tensor-copy destinations 128-byte aligned");

// Transpose of an 8 x 8 BF16 matrix held one 4-byte pair per lane (lane l:
// row l / 4, columns 2 (l % 4), 2 (l % 4) + 1), in the same layout.
__device__ __forceinline__ uint32_t movm_t(uint32_t a)
{
    uint32_t d;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
    return d;
}

// Four 8 x 8 BF16 matrices from shared memory, transposed (lanes 8j..8j+7
// give the 16-byte rows of matrix j).
__device__ __forceinline__ void ldsm_t4(uint32_t addr, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

struct WtTile {
    int b, x0, y0, z0;
};

__device__ __forceinline__ WtTile wt_tile(long long tile, int ntx, int nty, int ntz)
{
    long long q = tile;
    const int tx = (int)(q % ntx);
    q /= ntx;
    const int ty = (int)(q % nty);
    q /= nty;
    const int tz = (int)(q % ntz);
    return WtTile{(int)(q / ntz), tx * WT_TX, ty * WT_TY, tz * WT_TZ};
}

__global__ void __launch_bounds__(WT_THREADS, 1)
k_wgrad_tc(const __grid_constant__ CUtensorMap x_map, const __nv_bfloat16 *__restrict__ G, int B, int D, int H,
           int W, int ntx, int nty, int ntz, long long tiles, float *__restrict__ dW, float *__restrict__ db,
           int *fault)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sT = smem;                  // the three copies T_dx
    unsigned char *sG = smem + WT_OFF_G;       // G_T
    unsigned char *sX = smem + WT_OFF_X;       // X's halo tile, four 8-channel planes
    __shared__ __align__(8) uint64_t x_bar, mma_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        mbar_init(&x_bar, 1);
        mbar_init(&mma_bar, 1);
        mbar_init_fence();
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(WT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *abort_flag = &s_abort;
    const uint32_t *G2 = reinterpret_cast<const uint32_t *>(G);   // BF16 pairs
    const long long HW = (long long)H * W;
    const int r = lane >> 2, cp = lane & 3;   // the lane's row and channel pair in a G block
    const int cbg = warp & 3;                 // the warp's channel block of G
    float bs0 = 0.0f, bs1 = 0.0f;             // bias sums of channels 8 cbg + 2 cp, + 1
    // thread 0: X tiles copied / waited for, MMA batches committed / waited for
    int x_issued = 0, x_waited = 0, committed = 0, waited = 0;
    auto issue_x = [&](long long tile) {
        const WtTile t = wt_tile(tile, ntx, nty, ntz);
        mbar_expect_tx(&x_bar, 4 * WT_XPLANE);
        for (int cg = 0; cg < 4; cg++)
            asm volatile(
                "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];"
                ::"r"(smem_addr(sX + cg * WT_XPLANE)), "l"(reinterpret_cast<uint64_t>(&x_map)),
                  "r"(smem_addr(&x_bar)), "r"(cg * 8), "r"(t.x0 - 1), "r"(t.y0 - 1), "r"(t.z0 - 1), "r"(t.b)
                : "memory");
        x_issued++;
    };
    // the warp's 16 G blocks of a tile: pairs (row, kg) j = warp / 4 + 2 s, channel block cbg
    auto load_g = [&](long long tile, uint32_t (&v)[16]) {
        const WtTile t = wt_tile(tile, ntx, nty, ntz);
        const long long vb = HW * (long long)D * t.b;
#pragma unroll
        for (int s = 0; s < 16; s++) {
            const int j = (warp >> 2) + 2 * s;
            const int row = j >> 2, kg = j & 3;
            const int gx = t.x0 + 8 * kg + r, gy = t.y0 + row % WT_TY, gz = t.z0 + row / WT_TY;
            v[s] = 0u;   // voxels outside the volume add nothing
            if (gx < W && gy < H && gz < D)
                v[s] = __ldg(G2 + (((gx + (long long)W * gy + HW * gz + vb) * 32 + 8 * cbg) >> 1) + cp);
        }
    };
    uint32_t gv[16];
    long long tile = blockIdx.x;
    if (threadIdx.x == 0) issue_x(tile);
    load_g(tile, gv);
    for (int i = 0; tile < tiles; tile += gridDim.x, i++) {
        const bool okx = wait_or_abort(&x_bar, (uint32_t)(i & 1), abort_flag);
        if (threadIdx.x == 0 && okx) x_waited++;
        __syncthreads();
        if (*abort_flag) break;
        // ---- X -> T_dx: quad q = ((dx + 1) HZ + z') HY + y') 4 + cb, matrix j = K group
        const uint32_t xb = smem_addr(sX);
        for (int qd = warp; qd < WT_XQUADS; qd += WT_WARPS) {
            const int cb = qd & 3;
            int t = qd >> 2;
            const int yq = t % WT_HY;
            t /= WT_HY;
            const int zq = t % WT_HZ, dxi = t / WT_HZ;
            // halo x of interior x = 8 kg + row is 8 kg + row + 1 + dx
            const int hl = (zq * WT_HY + yq) * WT_HX + dxi + 8 * (lane >> 3) + (lane & 7);
            uint32_t v[4];
            ldsm_t4(xb + (uint32_t)(cb * WT_XPLANE + hl * 16), v);
            unsigned char *dst = sT + dxi * WT_COPY + ((zq * WT_HY + yq) * 4 + cb) * 128 + lane * 4;
#pragma unroll
            for (int kg = 0; kg < 4; kg++) *reinterpret_cast<uint32_t *>(dst + kg * WT_LBO) = v[kg];
        }
        // ---- G -> G_T (and the bias sums)
#pragma unroll
        for (int s = 0; s < 16; s++) {
            const int j = (warp >> 2) + 2 * s;
            bs0 += bf16_lo(gv[s]);
            bs1 += bf16_hi(gv[s]);
            *reinterpret_cast<uint32_t *>(sG + (j >> 2) * WT_GROW + (j & 3) * 512 + cbg * 128 + lane * 4) = movm_t(gv[s]);
        }
        fence_proxy_async_smem();   // generic stores, read next by the tensor cores
        __syncthreads();            // operands written, X's stage free
        const bool more = tile + gridDim.x < tiles;
        if (threadIdx.x == 0) {
            if (more) issue_x(tile + gridDim.x);   // lands while the MMAs run
            tc_fence_after();
            const uint32_t tb = smem_addr(sT), gb = smem_addr(sG);
            for (int c9 = 0; c9 < 9; c9++) {
                const int dz = c9 / 3 - 1, dxi = c9 % 3;
                const uint32_t d = tmem + (uint32_t)(c9 * 32);
                for (int iz = 0; iz < WT_TZ; iz++)
                    for (int iy = 0; iy < WT_TY; iy++) {
                        const int m0 = ((iz + 1 + dz) * WT_HY + iy) * 32;   // rows of dy = -1
                        for (int ks = 0; ks < 2; ks++) {
                            const uint64_t ad =
                                smem_desc(tb + (uint32_t)(dxi * WT_COPY + 2 * ks * WT_LBO + m0 * 16), WT_LBO, 128);
                            const uint64_t bd =
                                smem_desc(gb + (uint32_t)((iz * WT_TY + iy) * WT_GROW + 2 * ks * 512), 512, 128);
                            tc_mma(d, ad, bd, TcShape<32, 32>::IDESC, (committed | iz | iy | ks) ? 1u : 0u);
                        }
                    }
            }
            tc_commit(&mma_bar);
            committed++;
        }
        if (more) load_g(tile + gridDim.x, gv);   // in flight during the MMAs
        // the operands are rewritten only after the MMAs completed; the
        // barrier makes the decision to stop the same in every thread
        const bool ok = wait_or_abort(&mma_bar, (uint32_t)(i & 1), abort_flag);
        if (threadIdx.x == 0 && ok) waited++;
        tc_fence_after();
        __syncthreads();
        if (*abort_flag) break;
    }
    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) {
            atomicExch(fault, 1);
            // copies and MMA batches still in flight
            for (int j = x_waited; j < x_issued; j++) mbar_wait_bounded(&x_bar, (uint32_t)(j & 1), TC_WAIT_TRIES);
            for (int j = waited; j < committed; j++) mbar_wait_bounded(&mma_bar, (uint32_t)(j & 1), TC_WAIT_TRIES);
        }
    } else {
        if (warp < 3) {
            // TMEM lanes 32 warp + lane: dy = warp - 1, ci = lane
            for (int c9 = 0; c9 < 9; c9++) {
                float v[32];
                __syncwarp();
                tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(c9 * 32), v);
                const int tap = (c9 / 3) * 9 + warp * 3 + c9 % 3;
#pragma unroll
                for (int co = 0; co < 32; co++) atomicAdd(&dW[(long long)co * WT_KP + tap * 32 + lane], v[co]);
            }
        }
        // bias: sum over the 8 rows of a block (lanes with the same channel pair)
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            bs0 += __shfl_xor_sync(0xffffffffu, bs0, o);
            bs1 += __shfl_xor_sync(0xffffffffu, bs1, o);
        }
        if (db && lane < 4) {
            atomicAdd(&db[8 * cbg + 2 * lane], bs0);
            atomicAdd(&db[8 * cbg + 2 * lane + 1], bs1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    __syncwarp();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WT_TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------- host
static bool encode_activation_map(CUtensorMap *m, const void *in, int cin_mem, int B, int D, int H, int W,
                                  int bx = TC_HX, int by = TC_HY, int bz = TC_HZ)
{
    static void *fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        if (!fn) return false;
    }
    auto encode = reinterpret_cast<CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill)>(fn);
    const cuuint64_t row = (cuuint64_t)cin_mem * 2;   // bytes per voxel
    const cuuint64_t dims[5] = {(cuuint64_t)cin_mem, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B};
    const cuuint64_t strides[4] = {row, (cuuint64_t)W * row, (cuuint64_t)H * W * row, (cuuint64_t)D * H * W * row};
    const cuuint32_t box[5] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(in), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool conv3d_tc_available(const void *in, const void *Wb)
{
    return (reinterpret_cast<uintptr_t>(in) & 15u) == 0 && (reinterpret_cast<uintptr_t>(Wb) & 15u) == 0;
}

template <int CINP, int NOUT>
static cudaError_t launch_tc(cudaStream_t s, const CUtensorMap &map, const TcParams &p, int cin_mem, int out_ch,
                             const void *Wb, const float *bias, const void *res, void *out_b, float *out_f, int relu,
                             int *fault, int num_sms)
{
    using S = TcShape<CINP, NOUT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k_conv3d_tc<CINP, NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int grid = (int)(p.tiles < num_sms ? p.tiles : num_sms);
    k_conv3d_tc<CINP, NOUT><<<grid, TC_THREADS, S::SMEM, s>>>(
        p, map, cin_mem, out_ch, static_cast<const __nv_bfloat16 *>(Wb), bias, static_cast<const __nv_bfloat16 *>(res),
        static_cast<__nv_bfloat16 *>(out_b), out_f, relu, fault);
    return cudaGetLastError();
}

cudaError_t conv3d_tc(cudaStream_t s, int cin_mem, int cinp, int nout, int out_ch, const void *in, const void *Wb,
                      const float *bias, const void *res, void *out_b, float *out_f, int B, int D, int H, int W,
                      int relu, int *fault, int num_sms)
{
    if (!(cin_mem == 8 || cin_mem == 32) || cin_mem > cinp) return cudaErrorInvalidValue;
    if (out_ch > nout || (nout == 16 && (out_ch != 8 || res || out_b))) return cudaErrorInvalidValue;
    CUtensorMap map;
    if (!encode_activation_map(&map, in, cin_mem, B, D, H, W)) return cudaErrorInvalidValue;
    TcParams p;
    p.B = B;
    p.D = D;
    p.H = H;
    p.W = W;
    p.ntx = (W + TC_TX - 1) / TC_TX;
    p.nty = (H + TC_TY - 1) / TC_TY;
    p.ntz = (D + TC_TZ - 1) / TC_TZ;
    p.tiles = (long long)p.ntx * p.nty * p.ntz * B;
    if (cinp == 32 && nout == 32)
        return launch_tc<32, 32>(s, map, p, cin_mem, out_ch, Wb, bias, res, out_b, out_f, relu, fault, num_sms);
    if (cinp == 16 && nout == 32)
        return launch_tc<16, 32>(s, map, p, cin_mem, out_ch, Wb, bias, res, out_b, out_f, relu, fault, num_sms);
    if (cinp == 32 && nout == 16)
        return launch_tc<32, 16>(s, map, p, cin_mem, out_ch, Wb, bias, res, out_b, out_f, relu, fault, num_sms);
    return cudaErrorInvalidValue;
}

cudaError_t wgrad_tc32(cudaStream_t s, const void *X, const void *G, int B, int D, int H, int W, float *dW,
                       float *db, int *fault, int num_sms)
{
    if ((reinterpret_cast<uintptr_t>(X) & 15u) || (reinterpret_cast<uintptr_t>(G) & 3u) || !fault)
        return cudaErrorInvalidValue;
    CUtensorMap map;
    if (!encode_activation_map(&map, X, 32, B, D, H, W, WT_HX, WT_HY, WT_HZ)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, WT_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntx = (W + WT_TX - 1) / WT_TX, nty = (H + WT_TY - 1) / WT_TY, ntz = (D + WT_TZ - 1) / WT_TZ;
    const long long tiles = (long long)ntx * nty * ntz * B;
    if (tiles < 1) return cudaSuccess;
    const int grid = (int)(tiles < num_sms ? tiles : num_sms);
    k_wgrad_tc<<<grid, WT_THREADS, WT_SMEM, s>>>(map, static_cast<const __nv_bfloat16 *>(G), B, D, H, W, ntx, nty,
                                                ntz, tiles, dW, db, fault);
    return cudaGetLastError();
}

// Weights for the tensor-core kernel: dst[n][tap cinp + c] = src[n][tap cin + c]
// (src rows of kp_src), zero for n >= n_src or c >= cin.
__global__ void k_prep_tc_weights(const __nv_bfloat16 *__restrict__ src, int n_src, int cin, int kp_src, int nout,
                                  int cinp, __nv_bfloat16 *__restrict__ dst)
{
    const int total = nout * 27 * cinp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int n = e / (27 * cinp), k = e % (27 * cinp);
        const int tap = k / cinp, c = k % cinp;
        dst[e] = (n < n_src && c < cin) ? src[(size_t)n * kp_src + tap * cin + c] : __float2bfloat16(0.0f);
    }
}

void prep_tc_weights(cudaStream_t s, const void *src, int n_src, int cin, int kp_src, int nout, int cinp, void *dst)
{
    const int total = nout * 27 * cinp;
    k_prep_tc_weights<<<(total + 255) / 256, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(src), n_src, cin, kp_src,
                                                          nout, cinp, static_cast<__nv_bfloat16 *>(dst));
}

}  // namespace nn
}  // namespace rf
