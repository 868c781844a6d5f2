// noalloc.cu -- a Jacobi-PCG solve of the 7-point Picard system that
// allocates no device memory.
//
// Some callers cannot call cudaMalloc: host applications that own the
// device's memory through their own pool and forbid allocation once their
// time loop has started, coupled-model frameworks that must not trigger the
// implicit device synchronisation of cudaMalloc/cudaFree inside a step, and
// code that runs under a fixed memory budget decided at start-up.  For them
// this entry point keeps its work vectors in one file-scope device array of a
// fixed size; the caller passes only the operator, the right-hand side and the
// solution vector.
//
// The array is part of the library image: every GPU that loads the library
// holds it (3 343 104 bytes) until the process exits.  All calls share it, so
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race; callers must serialise them.  Each call clears the solver
// scalars, the reduction ticket and the launch counters before its first
// kernel and overwrites every vector entry it later reads, so nothing of a
// previous call's contents is read.
#include <algorithm>
#include <mutex>

#include "rf.h"
#include "rf_internal.cuh"

using namespace rf;

namespace {

constexpr long long NOALLOC_MAX_CELLS = RF_NOALLOC_MAX_CELLS;
constexpr int NOALLOC_MAX_BLOCKS = 2048;

// Layout of the scratch array (all offsets multiples of 256 bytes).
constexpr size_t VEC_BYTES = (size_t)NOALLOC_MAX_CELLS * sizeof(double);
constexpr size_t OFF_R = 0;
constexpr size_t OFF_Z = OFF_R + VEC_BYTES;
constexpr size_t OFF_P0 = OFF_Z + VEC_BYTES;
constexpr size_t OFF_P1 = OFF_P0 + VEC_BYTES;
constexpr size_t OFF_Q = OFF_P1 + VEC_BYTES;
constexpr size_t OFF_DINV = OFF_Q + VEC_BYTES;
constexpr size_t OFF_FLAGS = OFF_DINV + VEC_BYTES;
constexpr size_t OFF_PART = OFF_FLAGS + (((size_t)NOALLOC_MAX_CELLS + 255) & ~size_t(255));
constexpr size_t OFF_SCAL = OFF_PART + (size_t)8 * NOALLOC_MAX_BLOCKS * sizeof(double);
constexpr size_t OFF_TICKET = OFF_SCAL + 256;
constexpr size_t OFF_CTR = OFF_TICKET + 256;
constexpr size_t SCRATCH_BYTES = OFF_CTR + (((size_t)2 * KK_COUNT * sizeof(unsigned long long) + 255) & ~size_t(255));
static_assert(SCRATCH_BYTES == 3343104, "the scratch size stated in rf.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and cached.
std::mutex g_mutex;
constexpr int MAX_DEVICES = 64;
unsigned char *g_addr[MAX_DEVICES] = {nullptr};
int g_sms[MAX_DEVICES] = {0};

// dinv = 1/diag and the active flag (diag > 0) of every cell; clears the
// reduction ticket and the launch counters.
__global__ void k_noalloc_setup(long long N, const double *__restrict__ diag, double *__restrict__ dinv,
                                uint8_t *__restrict__ flags, unsigned int *ticket, unsigned long long *ctr)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) *ticket = 0u;
    if (t0 < 2 * KK_COUNT) ctr[t0] = 0ULL;
    for (long long p = t0; p < N; p += stride) {
        const double d = diag[p];
        const bool act = d > 0.0;
        dinv[p] = act ? 1.0 / d : 0.0;
        flags[p] = act ? FLAG_ACTIVE : 0;
    }
}

rf_status noalloc_fail(rf_status s, const char *msg)
{
    set_last_error(msg);
    return s;
}

}  // namespace

extern "C" rf_status rf_pcg_solve_noalloc(int nx, int ny, int nz, const double *d_diag, const double *d_Tx,
                                          const double *d_Ty, const double *d_Tz, const double *d_b, double *d_x,
                                          double tol, int max_it, void *cuda_stream, int *iters)
{
    if (nx < 1 || ny < 1 || nz < 1 || !d_diag || !d_Tx || !d_Ty || !d_Tz || !d_b || !d_x || !(tol > 0) || max_it < 1)
        return noalloc_fail(RF_ERR_ARG, "rf_pcg_solve_noalloc: invalid argument");
    const long long N = (long long)nx * ny * nz;
    if (N > NOALLOC_MAX_CELLS)
        return noalloc_fail(RF_ERR_ARG, "rf_pcg_solve_noalloc: more cells than RF_NOALLOC_MAX_CELLS");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return noalloc_fail(RF_ERR_NO_DEVICE, "rf_pcg_solve_noalloc: no usable CUDA device");
    unsigned char *base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            // the kernels are built for sm_103a only: refuse any other device
            // before the first launch (as rf_mesh_create does)
            int major = 0, minor = 0, nsm = 0;
            if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return noalloc_fail(RF_ERR_CUDA, "rf_pcg_solve_noalloc: device query failed");
            }
            if (major != 10 || minor != 3)
                return noalloc_fail(RF_ERR_NO_DEVICE, "rf_pcg_solve_noalloc: the device is not sm_103 (GB300)");
            void *ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return noalloc_fail(RF_ERR_CUDA, "rf_pcg_solve_noalloc: cudaGetSymbolAddress failed");
            }
            g_sms[dev] = nsm;
            g_addr[dev] = static_cast<unsigned char *>(ptr);
        }
        base = g_addr[dev];
        sms = g_sms[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    double *r = reinterpret_cast<double *>(base + OFF_R);
    double *z = reinterpret_cast<double *>(base + OFF_Z);
    double *p[2] = {reinterpret_cast<double *>(base + OFF_P0), reinterpret_cast<double *>(base + OFF_P1)};
    double *q = reinterpret_cast<double *>(base + OFF_Q);
    double *dinv = reinterpret_cast<double *>(base + OFF_DINV);
    uint8_t *flags = reinterpret_cast<uint8_t *>(base + OFF_FLAGS);
    double *partials = reinterpret_cast<double *>(base + OFF_PART);
    CgScal *sc = reinterpret_cast<CgScal *>(base + OFF_SCAL);
    unsigned int *ticket = reinterpret_cast<unsigned int *>(base + OFF_TICKET);
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(base + OFF_CTR);

    Grid g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.N = N;
    g.sxy = (long long)nx * ny;
    g.fx = make_fastdiv((unsigned int)nx);
    g.fxy = make_fastdiv((unsigned int)g.sxy);
    g.ctr = ctr;
    const long long want = (N + RED_THREADS - 1) / RED_THREADS;
    const int nblk = (int)std::max(1LL, std::min(want, std::min((long long)sms * 8, (long long)NOALLOC_MAX_BLOCKS)));
    const CondSet none{0, 0};

    // the scalars start from zero (done = 0) on every call; x0 is copied
    // into q (free until the first stencil product writes it) so that the
    // start kernel never reads the vector it writes
    if (cudaMemsetAsync(sc, 0, sizeof(CgScal), s) != cudaSuccess ||
        cudaMemcpyAsync(q, d_x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return noalloc_fail(RF_ERR_CUDA, "rf_pcg_solve_noalloc: CUDA error before the solve");
    k_noalloc_setup<<<nblk, RED_THREADS, 0, s>>>(N, d_diag, dinv, flags, ticket, ctr);
    launch_cg64_init(s, nblk, g, flags, q, d_x, d_b, d_Tx, d_Ty, d_Tz, d_diag, dinv, r, z, tol, max_it, partials,
                     ticket, sc, nullptr, none);
    if (cudaGetLastError() != cudaSuccess)
        return noalloc_fail(RF_ERR_CUDA, "rf_pcg_solve_noalloc: kernel launch failed");
    CgScal host{};
    long long launched = 0;
    int chunk = 2;
    for (;;) {
        for (int i = 0; i < chunk; i++, launched++) {
            double *pin = p[launched & 1], *pout = p[(launched + 1) & 1];
            launch_cg64_spmv(s, nblk, g, flags, z, pin, pout, q, d_Tx, d_Ty, d_Tz, d_diag, partials, ticket, sc);
            launch_cg64_update(s, nblk, g, d_x, r, z, pout, q, dinv, partials, ticket, sc, none);
        }
        if (cudaGetLastError() != cudaSuccess)
            return noalloc_fail(RF_ERR_CUDA, "rf_pcg_solve_noalloc: kernel launch failed");
        if (cudaMemcpyAsync(&host, sc, sizeof(CgScal), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return noalloc_fail(RF_ERR_CUDA, "rf_pcg_solve_noalloc: CUDA error during the solve");
        if (host.done) break;
        if (launched > (long long)max_it + 64)
            return noalloc_fail(RF_ERR_DEVICE_TIMEOUT, "rf_pcg_solve_noalloc: solve did not report completion");
        chunk = chunk < 64 ? 2 * chunk : 64;
    }
    if (iters) *iters = host.iter;
    if (host.status == CG_MAXIT) return noalloc_fail(RF_ERR_CG, "rf_pcg_solve_noalloc: max_it reached");
    if (host.status != CG_OK) return noalloc_fail(RF_ERR_CG, "rf_pcg_solve_noalloc: non-finite solve");
    return RF_OK;
}
