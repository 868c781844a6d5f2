// nn.cu -- kernels of the learned warm start: a 3-D convolutional residual
// network in BF16 with FP32 accumulation, trained on the GPU by these kernels.
//
// Layout: activations channels-last, [voxel][channel], voxel = x + W (y + H
// (z + D b)); channel counts padded to multiples of 8.  Weights of a layer:
// [Cout_p][K_p] with K = 27 Cin ordered (tap, channel), tap = (dz+1)*9 +
// (dy+1)*3 + (dx+1), zero-padded to K_p (a multiple of 16).
//
// Convolution = implicit GEMM: out[v][co] = sum_k A[v][k] W[co][k] with
// A[v][(tap, ci)] = in[v + tap][ci] (zero outside the volume).  Each warp
// computes 32 voxels x Cout with mma.sync.m16n8k16 (BF16 in, FP32 out),
// gathering A straight from global memory (pairs of channels per 32-bit
// load).  The input gradient is the same convolution with the transposed,
// tap-flipped weights; the weight gradient is a reduction over voxels done on
// the FP32 cores.
#include <cuda_bf16.h>

#include "nn.cuh"
#include "tma.cuh"

namespace rf {
namespace nn {

constexpr int CONV_WARPS = 4;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct Vox {
    int b, z, y, x;
    bool ok;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(CONV_WARPS * 32)
k_conv3d(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ Wp, const float *__restrict__ bias,
         const __nv_bfloat16 *__restrict__ res, __nv_bfloat16 *__restrict__ out_b, float *__restrict__ out_f,
         int B, int D, int H, int W, int relu)
{
    constexpr int K = 27 * CIN;
    constexpr int KP = (K + 15) / 16 * 16;
    constexpr int NT = COUT / 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long M = (long long)B * D * H * W;
    const long long m0 = ((long long)blockIdx.x * CONV_WARPS + warp) * 32;
    if (m0 >= M) return;
    Vox v[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        long long m = m0 + g + 8 * r;
        v[r].ok = m < M;
        if (!v[r].ok) m = 0;
        v[r].x = (int)(m % W);
        m /= W;
        v[r].y = (int)(m % H);
        m /= H;
        v[r].z = (int)(m % D);
        v[r].b = (int)(m / D);
    }
    float acc[2][NT][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < NT; j++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[i][j][e] = 0.0f;
    const unsigned *in32 = reinterpret_cast<const unsigned *>(in);
    const unsigned *w32 = reinterpret_cast<const unsigned *>(Wp);
    for (int kc = 0; kc < KP / 16; kc++) {
        unsigned av[4][2];   // [row r][half]
#pragma unroll
        for (int half = 0; half < 2; half++) {
            const int k = kc * 16 + 2 * t + 8 * half;
            const int tap = k / CIN, ci = k % CIN;
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int z = v[r].z + dz, y = v[r].y + dy, x = v[r].x + dx;
                const bool inb = v[r].ok && k < K && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W;
                unsigned val = 0u;
                if (inb) {
                    const long long vv = x + (long long)W * (y + (long long)H * (z + (long long)D * v[r].b));
                    val = __ldg(&in32[(vv * CIN + ci) >> 1]);
                }
                av[r][half] = val;
            }
        }
        unsigned a0[4] = {av[0][0], av[1][0], av[0][1], av[1][1]};
        unsigned a1[4] = {av[2][0], av[3][0], av[2][1], av[3][1]};
#pragma unroll
        for (int j = 0; j < NT; j++) {
            const int n = 8 * j + g;
            unsigned bf[2];
            bf[0] = __ldg(&w32[((long long)n * KP + kc * 16 + 2 * t) >> 1]);
            bf[1] = __ldg(&w32[((long long)n * KP + kc * 16 + 2 * t + 8) >> 1]);
            mma_bf16(acc[0][j], a0, bf);
            mma_bf16(acc[1][j], a1, bf);
        }
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < NT; j++)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const long long m = m0 + 16 * i + g + 8 * (e >> 1);
                if (m >= M) continue;
                const int col = 8 * j + 2 * t + (e & 1);
                float val = acc[i][j][e] + (bias ? bias[col] : 0.0f);
                if (res) val += __bfloat162float(res[m * COUT + col]);
                if (relu) val = fmaxf(val, 0.0f);
                if (out_b) out_b[m * COUT + col] = __float2bfloat16(val);
                if (out_f) out_f[m * COUT + col] = val;
            }
}


// Weight gradient of a convolution on the tensor cores (mma.sync m16n8k16,
// BF16 in, FP32 accumulate):
//   dW[co][tap CIN + ci] += sum_v G[v][co] X[v + off(tap)][ci],  db[co] += sum_v G[v][co].
// Blocks walk tiles of 32 x 4 x 2 voxels; the input tile with its halo
// (34 x 6 x 4) and the gradient tile sit in shared memory (64-byte rows with
// their 16-byte chunks XOR-swizzled so ldmatrix rows hit distinct banks;
// 16-byte rows are conflict-free as they are).  blockIdx.y selects one dz
// plane of 9 taps; warp w of the block owns tap (dz, w / 3 - 1, w % 3 - 1)
// and accumulates its COUT x CIN block in registers across all of the
// block's tiles; one atomic add per weight per block at the end.  K = 16
// consecutive x voxels of one (y, z) row per MMA; COUT = 8 uses the lower
// half of the M = 16 rows.
constexpr int WG_TX = 32, WG_TY = 4, WG_TZ = 2;
constexpr int WG_HX = WG_TX + 2, WG_HY = WG_TY + 2, WG_HZ = WG_TZ + 2;
constexpr int WG_HALO = WG_HX * WG_HY * WG_HZ;        // 816
constexpr int WG_INT = WG_TX * WG_TY * WG_TZ;          // 256
constexpr int WG_THREADS = 9 * 32;

// byte offset of 16-byte chunk `chunk` of row `row` in a tile of `chunks`-chunk rows
template <int CHUNKS>
__device__ __forceinline__ int wg_off(int row, int chunk)
{
    if constexpr (CHUNKS == 4) return row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4);
    else return row * 16;
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, unsigned (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, unsigned (&r)[2])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(addr));
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS)
k_wgrad_mma(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ G, int B, int D, int H, int W,
            long long tiles, int ntx, int nty, int ntz, float *__restrict__ dW, float *__restrict__ db)
{
    constexpr int XC = CIN / 8, GC = COUT / 8;        // 16-byte chunks per row
    constexpr int COB = COUT >= 16 ? COUT / 16 : 1;   // M = 16 blocks of output channels
    constexpr int CIB = CIN / 8;                      // N = 8 blocks of input channels
    constexpr int KP = (27 * CIN + 15) / 16 * 16;
    extern __shared__ __align__(128) unsigned char wg_smem[];
    unsigned char *sX = wg_smem;                       // WG_HALO rows of 16 XC bytes
    unsigned char *sG = wg_smem + WG_HALO * 16 * XC;   // WG_INT rows of 16 GC bytes
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, g = lane >> 2, t = lane & 3;
    const int dz = (int)blockIdx.y - 1, dy = warp / 3 - 1, dx = warp % 3 - 1;
    const int tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
    const int off = (dz * WG_HY + dy) * WG_HX + dx;
    float acc[COB][CIB][4];
#pragma unroll
    for (int a = 0; a < COB; a++)
#pragma unroll
        for (int b = 0; b < CIB; b++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[a][b][e] = 0.0f;
    float accb = 0.0f;   // bias gradient of channel threadIdx.x (dz = 0 blocks, threads < COUT)
    const uint32_t sXa = smem_addr(sX), sGa = smem_addr(sG);
    const long long HW = (long long)H * W;
    const int mtx = lane >> 3, rr = lane & 7;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        long long r = tile;
        const int tx = (int)(r % ntx);
        r /= ntx;
        const int ty = (int)(r % nty);
        r /= nty;
        const int tz = (int)(r % ntz);
        const int b = (int)(r / ntz);
        const int x0 = tx * WG_TX, y0 = ty * WG_TY, z0 = tz * WG_TZ;
        __syncthreads();   // the previous tile's shared data is no longer read
        for (int e = threadIdx.x; e < WG_HALO * XC; e += WG_THREADS) {
            const int row = e / XC, ch = e % XC;
            const int hx = row % WG_HX, hy = (row / WG_HX) % WG_HY, hz = row / (WG_HX * WG_HY);
            const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (x >= 0 && x < W && y >= 0 && y < H && z >= 0 && z < D)
                v = __ldg(reinterpret_cast<const uint4 *>(X + (x + (long long)W * y + HW * (z + (long long)D * b)) * CIN) + ch);
            *reinterpret_cast<uint4 *>(sX + wg_off<XC>(row, ch)) = v;
        }
        for (int e = threadIdx.x; e < WG_INT * GC; e += WG_THREADS) {
            const int row = e / GC, ch = e % GC;
            const int ix = row % WG_TX, iy = (row / WG_TX) % WG_TY, iz = row / (WG_TX * WG_TY);
            const int x = x0 + ix, y = y0 + iy, z = z0 + iz;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);   // voxels outside the volume add nothing
            if (x < W && y < H && z < D)
                v = __ldg(reinterpret_cast<const uint4 *>(G + (x + (long long)W * y + HW * (z + (long long)D * b)) * COUT) + ch);
            *reinterpret_cast<uint4 *>(sG + wg_off<GC>(row, ch)) = v;
        }
        __syncthreads();
        if (dz == 0 && threadIdx.x < COUT && db) {
            for (int row = 0; row < WG_INT; row++) {
                const __nv_bfloat16 *gr = reinterpret_cast<const __nv_bfloat16 *>(sG + wg_off<GC>(row, threadIdx.x >> 3));
                accb += __bfloat162float(gr[threadIdx.x & 7]);
            }
        }
        // 16 K-steps: (iz, iy) rows x two halves of 16 x voxels
        for (int ks = 0; ks < WG_INT / 16; ks++) {
            const int iv0 = ks * 16;                                    // interior row of the first voxel
            const int ix0 = iv0 % WG_TX, iy = (iv0 / WG_TX) % WG_TY, iz = iv0 / (WG_TX * WG_TY);
            const int hl0 = ((iz + 1) * WG_HY + (iy + 1)) * WG_HX + (ix0 + 1) + off;   // shifted input row
            // A = G^T (co x v): matrices (co lo, v 0-7), (co hi, v 0-7), (co lo, v 8-15), (co hi, v 8-15)
            unsigned af[COB][4];
            if constexpr (COUT >= 16) {
#pragma unroll
                for (int cb = 0; cb < COB; cb++)
                    ldsm_x4_t(sGa + wg_off<GC>(iv0 + rr + ((mtx >> 1) << 3), 2 * cb + (mtx & 1)), af[cb]);
            } else {
                unsigned a2[2];   // co 0-7 only; rows 8-15 of the M = 16 block are zero
                ldsm_x2_t(sGa + wg_off<GC>(iv0 + rr + ((mtx & 1) << 3), 0), a2);
                af[0][0] = a2[0];
                af[0][1] = 0u;
                af[0][2] = a2[1];
                af[0][3] = 0u;
            }
            // B = X shift (v x ci): matrices (v 0-7, ci blk j), (v 8-15, ci blk j), (v 0-7, j+1), (v 8-15, j+1)
            if constexpr (CIB >= 2) {
#pragma unroll
                for (int jb = 0; jb < CIB / 2; jb++) {
                    unsigned bf[4];
                    ldsm_x4_t(sXa + wg_off<XC>(hl0 + rr + ((mtx & 1) << 3), 2 * jb + (mtx >> 1)), bf);
#pragma unroll
                    for (int cb = 0; cb < COB; cb++) {
                        const unsigned b0[2] = {bf[0], bf[1]}, b1[2] = {bf[2], bf[3]};
                        mma_bf16(acc[cb][2 * jb], af[cb], b0);
                        mma_bf16(acc[cb][2 * jb + 1], af[cb], b1);
                    }
                }
            } else {
                unsigned bf[2];
                ldsm_x2_t(sXa + wg_off<XC>(hl0 + rr + ((mtx & 1) << 3), 0), bf);
#pragma unroll
                for (int cb = 0; cb < COB; cb++) mma_bf16(acc[cb][0], af[cb], bf);
            }
        }
    }
    // one atomic add per weight (and per bias) per block
#pragma unroll
    for (int cb = 0; cb < COB; cb++)
#pragma unroll
        for (int j = 0; j < CIB; j++)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int co = 16 * cb + g + 8 * (e >> 1), ci = 8 * j + 2 * t + (e & 1);
                if (co < COUT) atomicAdd(&dW[(long long)co * KP + tap * CIN + ci], acc[cb][j][e]);
            }
    if (dz == 0 && threadIdx.x < COUT && db) atomicAdd(&db[threadIdx.x], accb);
}

__global__ void k_relu_bwd(const __nv_bfloat16 *__restrict__ y, const float *__restrict__ dy, float *__restrict__ dx,
                           long long n, const float *__restrict__ add)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float g = __bfloat162float(y[i]) > 0.0f ? dy[i] : 0.0f;
        if (add) g += add[i];
        dx[i] = g;
    }
}

__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

__global__ void k_add(float *__restrict__ a, const float *__restrict__ b, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] += b[i];
}

// channel 0 of pred [M][8] against target [M] with a mask [M] (0/1):
// L += (mask (pred - target))^2 / count, dpred = 2 mask^2 (pred - target) / count
__global__ void k_mse(const float *__restrict__ pred, const float *__restrict__ target,
                      const float *__restrict__ mask, long long M, float inv_count, float *__restrict__ dpred,
                      float *__restrict__ loss)
{
    float s = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
        const float w = mask ? mask[i] : 1.0f;
        const float d = (pred[i * 8] - target[i]) * w;
        s = fmaf(d, d, s);
        dpred[i * 8] = 2.0f * d * w * inv_count;
#pragma unroll
        for (int c = 1; c < 8; c++) dpred[i * 8 + c] = 0.0f;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_count);
}

// Adam (Kingma & Ba 2015) on FP32 master weights.
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// BF16 weights for the forward conv and the transposed, tap-flipped weights
// for the input gradient: Wt[ci][tap' COUT + co] = W[co][tap CIN + ci],
// tap' = 26 - tap.
__global__ void k_prep_weights(const float *__restrict__ W, int Cinp, int Coutp, int KP, int KPt,
                               __nv_bfloat16 *__restrict__ Wb, __nv_bfloat16 *__restrict__ Wt)
{
    const int K = 27 * Cinp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Coutp * KP; i += gridDim.x * blockDim.x) {
        const int co = i / KP, k = i % KP;
        const float val = W[i];
        Wb[i] = __float2bfloat16(val);
        if (Wt && k < K) {
            const int tap = k / Cinp, ci = k % Cinp;
            Wt[(long long)ci * KPt + (26 - tap) * Coutp + co] = __float2bfloat16(val);
        }
    }
}

// FP32 features [M][4] -> BF16 [M][8], channels 4..7 zero.
__global__ void k_pad_features(const float4 *__restrict__ x4, uint4 *__restrict__ x8, long long M)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
        const float4 f = x4[i];
        const __nv_bfloat162 lo = __floats2bfloat162_rn(f.x, f.y), hi = __floats2bfloat162_rn(f.z, f.w);
        uint4 o;
        o.x = *reinterpret_cast<const unsigned *>(&lo);
        o.y = *reinterpret_cast<const unsigned *>(&hi);
        o.z = 0u;
        o.w = 0u;
        x8[i] = o;
    }
}

// ------------------------------------------------------------ solver side
// Network inputs of cell p: h / h_scale; (ln Ks - mean) / std; the top
// boundary flux feature on cells that carry the top face; ln(dt / t_scale).
// Inactive cells are all zero (the network sees them like its padding).
__device__ __forceinline__ float4 ws_feature(uint8_t fl, double h, double Ks, const WsScales &sc, float q_feat,
                                             float dt_feat)
{
    if (!(fl & FLAG_ACTIVE)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float4 f;
    f.x = (float)(h / sc.h_scale);
    f.y = (float)((log(Ks) - sc.lnK_mean) / sc.lnK_std);
    f.z = (fl & (1u << F_ZMAX)) ? q_feat : 0.0f;
    f.w = dt_feat;
    return f;
}

__global__ void k_ws_features_f32(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ h,
                                  const double *__restrict__ Ks, WsScales sc, float q_feat, float dt_feat,
                                  float4 *__restrict__ out)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += (long long)gridDim.x * blockDim.x)
        out[p] = ws_feature(flags[p], h[p], Ks[p], sc, q_feat, dt_feat);
}

__global__ void k_ws_features_bf16(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ h,
                                   const double *__restrict__ Ks, WsScales sc, float q_feat, float dt_feat,
                                   uint4 *__restrict__ out)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += (long long)gridDim.x * blockDim.x) {
        const float4 f = ws_feature(flags[p], h[p], Ks[p], sc, q_feat, dt_feat);
        const __nv_bfloat162 lo = __floats2bfloat162_rn(f.x, f.y), hi = __floats2bfloat162_rn(f.z, f.w);
        uint4 o;
        o.x = *reinterpret_cast<const unsigned *>(&lo);
        o.y = *reinterpret_cast<const unsigned *>(&hi);
        o.z = 0u;
        o.w = 0u;
        out[p] = o;
    }
}

// hk = h + y scale on active cells (scale = out_scale dt); h where y is not finite.
__global__ void k_ws_guess(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ h,
                           const float *__restrict__ y, double scale, double *__restrict__ hk)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += (long long)gridDim.x * blockDim.x) {
        const float yp = y[p * C_OUT_P];
        double v = h[p];
        if ((flags[p] & FLAG_ACTIVE) && isfinite(yp)) v += (double)yp * scale;
        hk[p] = v;
    }
}

// target = (h_new - h_old) / (out_scale dt), mask = 1 on active cells.
__global__ void k_ws_target(Grid g, const uint8_t *__restrict__ flags, const double *__restrict__ hn1,
                            const double *__restrict__ hn, double inv_scale, float *__restrict__ target,
                            float *__restrict__ mask)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += (long long)gridDim.x * blockDim.x) {
        const bool act = flags[p] & FLAG_ACTIVE;
        target[p] = act ? (float)((hn1[p] - hn[p]) * inv_scale) : 0.0f;
        if (mask) mask[p] = act ? 1.0f : 0.0f;
    }
}

// ---------------------------------------------------------------- launchers
static int nblocks(long long n, int t) { return (int)((n + t - 1) / t > 4096 ? 4096 : (n + t - 1) / t); }

cudaError_t conv3d(cudaStream_t s, int cin, int cout, const void *in, const void *Wb, const float *bias,
                   const void *res, void *out_b, float *out_f, int B, int D, int H, int W, int relu)
{
    const long long M = (long long)B * D * H * W;
    const int grid = (int)((M + 32 * CONV_WARPS - 1) / (32 * CONV_WARPS));
    auto i = static_cast<const __nv_bfloat16 *>(in);
    auto w = static_cast<const __nv_bfloat16 *>(Wb);
    auto r = static_cast<const __nv_bfloat16 *>(res);
    auto ob = static_cast<__nv_bfloat16 *>(out_b);
    if (cin == 8 && cout == 32) k_conv3d<8, 32><<<grid, 32 * CONV_WARPS, 0, s>>>(i, w, bias, r, ob, out_f, B, D, H, W, relu);
    else if (cin == 32 && cout == 32) k_conv3d<32, 32><<<grid, 32 * CONV_WARPS, 0, s>>>(i, w, bias, r, ob, out_f, B, D, H, W, relu);
    else if (cin == 32 && cout == 8) k_conv3d<32, 8><<<grid, 32 * CONV_WARPS, 0, s>>>(i, w, bias, r, ob, out_f, B, D, H, W, relu);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t launch_wgrad_mma(cudaStream_t s, const void *X, const void *G, int B, int D, int H, int W,
                                    float *dW, float *db, int num_sms)
{
    const int ntx = (W + WG_TX - 1) / WG_TX, nty = (H + WG_TY - 1) / WG_TY, ntz = (D + WG_TZ - 1) / WG_TZ;
    const long long tiles = (long long)ntx * nty * ntz * B;
    const long long want = 2LL * num_sms;   // x 3 dz planes
    dim3 grid((unsigned)(tiles < want ? tiles : want), 3);
    constexpr int smem = WG_HALO * 2 * CIN + WG_INT * 2 * COUT;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad_mma<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_wgrad_mma<CIN, COUT><<<grid, WG_THREADS, smem, s>>>(static_cast<const __nv_bfloat16 *>(X),
                                                          static_cast<const __nv_bfloat16 *>(G), B, D, H, W, tiles,
                                                          ntx, nty, ntz, dW, db);
    return cudaGetLastError();
}

cudaError_t wgrad_mma(cudaStream_t s, int cin, int cout, const void *X, const void *G, int B, int D, int H, int W,
                      float *dW, float *db, int num_sms)
{
    if (cin == 32 && cout == 32) return launch_wgrad_mma<32, 32>(s, X, G, B, D, H, W, dW, db, num_sms);
    if (cin == 8 && cout == 32) return launch_wgrad_mma<8, 32>(s, X, G, B, D, H, W, dW, db, num_sms);
    if (cin == 32 && cout == 8) return launch_wgrad_mma<32, 8>(s, X, G, B, D, H, W, dW, db, num_sms);
    return cudaErrorInvalidValue;
}

void relu_bwd(cudaStream_t s, const void *y, const float *dy, float *dx, long long n, const float *add)
{
    k_relu_bwd<<<nblocks(n, 256), 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(y), dy, dx, n, add);
}
void to_bf16(cudaStream_t s, const float *a, void *b, long long n)
{
    k_to_bf16<<<nblocks(n, 256), 256, 0, s>>>(a, static_cast<__nv_bfloat16 *>(b), n);
}
void add(cudaStream_t s, float *a, const float *b, long long n) { k_add<<<nblocks(n, 256), 256, 0, s>>>(a, b, n); }
void mse(cudaStream_t s, const float *pred, const float *target, const float *mask, long long M, float inv_count,
         float *dpred, float *loss)
{
    k_mse<<<nblocks(M, 256), 256, 0, s>>>(pred, target, mask, M, inv_count, dpred, loss);
}
void adam(cudaStream_t s, float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
          float eps, float c1, float c2)
{
    k_adam<<<nblocks(n, 256), 256, 0, s>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
}
void prep_weights(cudaStream_t s, const float *W, int Cinp, int Coutp, int KP, int KPt, void *Wb, void *Wt)
{
    k_prep_weights<<<nblocks((long long)Coutp * KP, 256), 256, 0, s>>>(
        W, Cinp, Coutp, KP, KPt, static_cast<__nv_bfloat16 *>(Wb), static_cast<__nv_bfloat16 *>(Wt));
}

void pad_features(cudaStream_t s, const float *x4, void *x8, long long M)
{
    k_pad_features<<<nblocks(M, 256), 256, 0, s>>>(reinterpret_cast<const float4 *>(x4), static_cast<uint4 *>(x8), M);
}

void ws_features_f32(cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h, const double *Ks,
                     const WsScales &sc, float q_feat, float dt_feat, float *out)
{
    k_ws_features_f32<<<nblocks(g.N, 256), 256, 0, s>>>(g, flags, h, Ks, sc, q_feat, dt_feat,
                                                        reinterpret_cast<float4 *>(out));
}

void ws_features_bf16(cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h, const double *Ks,
                      const WsScales &sc, float q_feat, float dt_feat, void *out)
{
    k_ws_features_bf16<<<nblocks(g.N, 256), 256, 0, s>>>(g, flags, h, Ks, sc, q_feat, dt_feat,
                                                         static_cast<uint4 *>(out));
}

void ws_guess(cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h, const float *y, double scale,
              double *hk)
{
    k_ws_guess<<<nblocks(g.N, 256), 256, 0, s>>>(g, flags, h, y, scale, hk);
}

void ws_target(cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h_new, const double *h_old,
               double inv_scale, float *target, float *mask)
{
    k_ws_target<<<nblocks(g.N, 256), 256, 0, s>>>(g, flags, h_new, h_old, inv_scale, target, mask);
}

}  // namespace nn
}  // namespace rf
