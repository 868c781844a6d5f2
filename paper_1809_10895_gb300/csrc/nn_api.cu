// nn_api.cu -- the warm-start network object behind the rf_nn_* C ABI:
// parameter storage (FP32 master copy, BF16 forward and transposed copies,
// Adam moments), activation workspaces, and the forward / backward / update
// sequences of kernels from nn.cu.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "nn.cuh"
#include "rf.h"

using namespace rf;

namespace {

struct LayerDims {
    int cin, cout;       // logical channels
    int cinp, coutp;     // padded channels
    int kp, kpt;         // padded reduction lengths of the forward / transposed weights
    long long w, b;      // offsets of W[coutp][kp] and b[coutp] in the FP32 parameter buffer
    long long wb, wt;    // offsets in the BF16 forward / transposed weight buffers
};

}  // namespace

struct rf_nn {
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    rf_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> allocations;
    cudaEvent_t ev = nullptr;   // completion of the network's last piece of work

    LayerDims L[nn::N_LAYERS];
    long long nP = 0, nWb = 0, nWt = 0;
    float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr;
    __nv_bfloat16 *Wb = nullptr, *Wt = nullptr;
    // tensor-core layouts of the input and output convolutions (channels
    // padded to the MMA's K = 16 and N = 16 granules)
    __nv_bfloat16 *tcw0 = nullptr, *tcw9 = nullptr, *tcw9t = nullptr;
    float *loss_d = nullptr, *loss_h = nullptr;
    int *fault = nullptr, *fault_h = nullptr;   // set by a device wait that ran out
    int adam_t = 0;
    long long launches = 0;

    // inference workspace (voxels)
    long long cap_inf = 0;
    __nv_bfloat16 *ix = nullptr, *iA = nullptr, *iU = nullptr, *iA2 = nullptr;
    float *iy = nullptr;
    // training workspace
    long long cap_tr = 0;
    __nv_bfloat16 *tx = nullptr, *ta[5] = {}, *tu[4] = {}, *tdyb = nullptr, *tgb = nullptr;
    float *ty = nullptr, *tdy = nullptr, *tgA = nullptr, *tgB = nullptr, *tgC = nullptr;
    // trace of the last gradient evaluation (rf_nn_set_trace): the BF16
    // output gradient of every layer, kept as each layer's weight gradient
    // and input gradient read it
    bool trace = false;
    long long trace_cap = 0, trace_M = 0;
    __nv_bfloat16 *trace_g[nn::N_LAYERS] = {};

    void *dalloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        void *p = nullptr;
        if (has_alloc) p = alloc.alloc(bytes, alloc.user);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        if (p) allocations.push_back(p);
        return p;
    }
    void dfree(void *p)
    {
        if (!p) return;
        for (size_t i = 0; i < allocations.size(); i++)
            if (allocations[i] == p) {
                allocations.erase(allocations.begin() + (long)i);
                break;
            }
        if (has_alloc) alloc.free(p, alloc.user);
        else cudaFree(p);
    }
};

namespace {

rf_status nfail(rf_status s, const std::string &msg)
{
    rf::set_last_error(msg.c_str());
    return s;
}

#define NN_CUDA(x)                                                                              \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) return nfail(RF_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define NN_TRY(x)                      \
    do {                               \
        rf_status s_ = (x);            \
        if (s_ != RF_OK) return s_;    \
    } while (0)

template <class T>
bool nalloc(rf_nn *n, T *&p, long long count)
{
    p = static_cast<T *>(n->dalloc(sizeof(T) * (size_t)(count > 0 ? count : 1)));
    return p != nullptr;
}

void layout(rf_nn *n)
{
    long long off = 0, ob = 0, ot = 0;
    for (int l = 0; l < nn::N_LAYERS; l++) {
        LayerDims &d = n->L[l];
        d.cin = l == 0 ? nn::C_IN : nn::C_HID;
        d.cout = l == nn::N_LAYERS - 1 ? nn::C_OUT : nn::C_HID;
        d.cinp = l == 0 ? nn::C_IN_P : nn::C_HID;
        d.coutp = l == nn::N_LAYERS - 1 ? nn::C_OUT_P : nn::C_HID;
        d.kp = nn::round16(27 * d.cinp);
        d.kpt = nn::round16(27 * d.coutp);
        d.w = off;
        off += (long long)d.coutp * d.kp;
        d.b = off;
        off += d.coutp;
        d.wb = ob;
        ob += (long long)d.coutp * d.kp;
        d.wt = ot;
        ot += (long long)d.cinp * d.kpt;
    }
    n->nP = off;
    n->nWb = ob;
    n->nWt = ot;
}

// Order this work after the network's previous work (on any stream).
rf_status begin(rf_nn *n, cudaStream_t s)
{
    NN_CUDA(cudaStreamWaitEvent(s, n->ev, 0));
    return RF_OK;
}
rf_status end(rf_nn *n, cudaStream_t s)
{
    NN_CUDA(cudaGetLastError());
    NN_CUDA(cudaEventRecord(n->ev, s));
    return RF_OK;
}

rf_status refresh_weights(rf_nn *n, cudaStream_t s)
{
    for (int l = 0; l < nn::N_LAYERS; l++) {
        const LayerDims &d = n->L[l];
        nn::prep_weights(s, n->P + d.w, d.cinp, d.coutp, d.kp, d.kpt, n->Wb + d.wb, l == 0 ? nullptr : n->Wt + d.wt);
        n->launches++;
    }
    const LayerDims &d0 = n->L[0], &d9 = n->L[nn::N_LAYERS - 1];
    nn::prep_tc_weights(s, n->Wb + d0.wb, d0.coutp, d0.cinp, d0.kp, 32, 16, n->tcw0);     // 8 -> 32
    nn::prep_tc_weights(s, n->Wb + d9.wb, d9.coutp, d9.cinp, d9.kp, 16, 32, n->tcw9);     // 32 -> 8 (N 16)
    nn::prep_tc_weights(s, n->Wt + d9.wt, d9.cinp, d9.coutp, d9.kpt, 32, 16, n->tcw9t);   // its input gradient
    n->launches += 3;
    return RF_OK;
}

rf_status ensure_inference(rf_nn *n, long long M)
{
    if (M <= n->cap_inf) return RF_OK;
    for (void *p : {(void *)n->ix, (void *)n->iA, (void *)n->iU, (void *)n->iA2, (void *)n->iy}) n->dfree(p);
    n->cap_inf = 0;
    if (!(nalloc(n, n->ix, M * nn::C_IN_P) && nalloc(n, n->iA, M * nn::C_HID) && nalloc(n, n->iU, M * nn::C_HID) &&
          nalloc(n, n->iA2, M * nn::C_HID) && nalloc(n, n->iy, M * nn::C_OUT_P)))
        return nfail(RF_ERR_NOMEM, "warm-start network: inference workspace allocation failed");
    n->cap_inf = M;
    return RF_OK;
}

rf_status ensure_training(rf_nn *n, long long M)
{
    if (M <= n->cap_tr) return RF_OK;
    std::vector<void *> old = {n->tx, n->tdyb, n->tgb, n->ty, n->tdy, n->tgA, n->tgB, n->tgC};
    for (auto p : n->ta) old.push_back(p);
    for (auto p : n->tu) old.push_back(p);
    for (void *p : old) n->dfree(p);
    n->cap_tr = 0;
    bool ok = nalloc(n, n->tx, M * nn::C_IN_P) && nalloc(n, n->tdyb, M * nn::C_OUT_P) &&
              nalloc(n, n->tgb, M * nn::C_HID) && nalloc(n, n->ty, M * nn::C_OUT_P) &&
              nalloc(n, n->tdy, M * nn::C_OUT_P) && nalloc(n, n->tgA, M * nn::C_HID) &&
              nalloc(n, n->tgB, M * nn::C_HID) && nalloc(n, n->tgC, M * nn::C_HID);
    for (int i = 0; i < 5 && ok; i++) ok = nalloc(n, n->ta[i], M * nn::C_HID);
    for (int i = 0; i < 4 && ok; i++) ok = nalloc(n, n->tu[i], M * nn::C_HID);
    if (!ok) return nfail(RF_ERR_NOMEM, "warm-start network: training workspace allocation failed");
    n->cap_tr = M;
    return RF_OK;
}

rf_status conv(rf_nn *n, cudaStream_t s, int l, bool transposed, const void *in, const void *res, void *out_b,
               float *out_f, int B, int D, int H, int W, int relu, int *fault = nullptr)
{
    const LayerDims &d = n->L[l];
    cudaError_t e;
    const void *w = transposed ? (const void *)(n->Wt + d.wt) : (const void *)(n->Wb + d.wb);
    int *f = fault ? fault : n->fault;
    const bool last = l == nn::N_LAYERS - 1;
    // every layer shape of the network runs on the tcgen05 tensor cores
    if (d.cinp == 32 && d.coutp == 32 && nn::conv3d_tc_available(in, w)) {
        e = nn::conv3d_tc(s, 32, 32, 32, 32, in, w, transposed ? nullptr : n->P + d.b, transposed ? nullptr : res,
                          out_b, out_f, B, D, H, W, transposed ? 0 : relu, f, n->num_sms);
        n->launches++;
        NN_CUDA(e);
        return RF_OK;
    }
    if (l == 0 && !transposed && nn::conv3d_tc_available(in, n->tcw0)) {
        e = nn::conv3d_tc(s, 8, 16, 32, 32, in, n->tcw0, n->P + d.b, res, out_b, out_f, B, D, H, W, relu, f,
                          n->num_sms);
        n->launches++;
        NN_CUDA(e);
        return RF_OK;
    }
    if (last && !transposed && !out_b && !res && nn::conv3d_tc_available(in, n->tcw9)) {
        e = nn::conv3d_tc(s, 32, 32, 16, 8, in, n->tcw9, n->P + d.b, nullptr, nullptr, out_f, B, D, H, W, relu, f,
                          n->num_sms);
        n->launches++;
        NN_CUDA(e);
        return RF_OK;
    }
    if (last && transposed && nn::conv3d_tc_available(in, n->tcw9t)) {
        e = nn::conv3d_tc(s, 8, 16, 32, 32, in, n->tcw9t, nullptr, nullptr, out_b, out_f, B, D, H, W, 0, f,
                          n->num_sms);
        n->launches++;
        NN_CUDA(e);
        return RF_OK;
    }
    if (!transposed)
        e = nn::conv3d(s, d.cinp, d.coutp, in, n->Wb + d.wb, n->P + d.b, res, out_b, out_f, B, D, H, W, relu);
    else
        e = nn::conv3d(s, d.coutp, d.cinp, in, n->Wt + d.wt, nullptr, nullptr, out_b, out_f, B, D, H, W, 0);
    n->launches++;
    NN_CUDA(e);
    return RF_OK;
}

// Forward pass from BF16 padded features x (M x 8) into y (M x 8, FP32).
// Inference ping-pongs three M x 32 BF16 buffers; training keeps every
// activation for the backward pass.
rf_status forward(rf_nn *n, cudaStream_t s, const void *x, int B, int D, int H, int W, float *y, bool train,
                  int *fault = nullptr)
{
    __nv_bfloat16 *A = train ? n->ta[0] : n->iA;
    NN_TRY(conv(n, s, 0, false, x, nullptr, A, nullptr, B, D, H, W, 1));
    for (int blk = 0; blk < 4; blk++) {
        __nv_bfloat16 *U = train ? n->tu[blk] : n->iU;
        __nv_bfloat16 *A2 = train ? n->ta[blk + 1] : n->iA2;
        NN_TRY(conv(n, s, 1 + 2 * blk, false, A, nullptr, U, nullptr, B, D, H, W, 1, fault));
        NN_TRY(conv(n, s, 2 + 2 * blk, false, U, A, A2, nullptr, B, D, H, W, 1, fault));
        if (train) A = A2;
        else std::swap(n->iA, n->iA2), A = n->iA;
    }
    NN_TRY(conv(n, s, 9, false, A, nullptr, nullptr, y, B, D, H, W, 0));
    return RF_OK;
}

__global__ void k_take0(const float *__restrict__ y8, float *__restrict__ y, long long M)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
        y[i] = y8[i * nn::C_OUT_P];
}

// Weight gradient of a layer from its BF16 input and BF16 output gradient, on
// the tensor cores: tcgen05 for the 32 -> 32 layers, mma.sync for the input
// and output layers (8 padded channels on one side).
rf_status wgrad_tc(rf_nn *n, cudaStream_t s, int l, const void *in, const void *g_bf16, int B, int D, int H, int W)
{
    const LayerDims &d = n->L[l];
    n->launches++;
    if (d.cinp == 32 && d.coutp == 32)
        NN_CUDA(nn::wgrad_tc32(s, in, g_bf16, B, D, H, W, n->G + d.w, n->G + d.b, n->fault, n->num_sms));
    else
        NN_CUDA(nn::wgrad_mma(s, d.cinp, d.coutp, in, g_bf16, B, D, H, W, n->G + d.w, n->G + d.b, n->num_sms));
    return RF_OK;
}

// Loss and gradient (into n->G, padded layout); the loss lands in n->loss_d.
rf_status loss_grad(rf_nn *n, const float *x4, const float *target, const float *mask, int B, int D, int H, int W)
{
    cudaStream_t s = n->stream;
    const long long M = (long long)B * D * H * W;
    NN_TRY(ensure_training(n, M));
    nn::pad_features(s, x4, n->tx, M);
    n->launches++;
    NN_TRY(forward(n, s, n->tx, B, D, H, W, n->ty, true));
    NN_CUDA(cudaMemsetAsync(n->loss_d, 0, sizeof(float), s));
    nn::mse(s, n->ty, target, mask, M, (float)(1.0 / (double)M), n->tdy, n->loss_d);
    NN_CUDA(cudaMemsetAsync(n->G, 0, sizeof(float) * n->nP, s));
    const long long MH = M * nn::C_HID;
    // output convolution
    if (n->trace && n->trace_cap < M) {
        for (auto &p : n->trace_g) {
            n->dfree(p);
            p = nullptr;
        }
        n->trace_cap = 0;
        for (int l = 0; l < nn::N_LAYERS; l++)
            if (!nalloc(n, n->trace_g[l], M * nn::C_HID))
                return nfail(RF_ERR_NOMEM, "warm-start network: trace allocation failed");
        n->trace_cap = M;
    }
    // keep the BF16 output gradient of layer l (M x channels) for the trace
    auto keep = [&](int l, const __nv_bfloat16 *src, long long count) -> rf_status {
        if (n->trace)
            NN_CUDA(cudaMemcpyAsync(n->trace_g[l], src, sizeof(__nv_bfloat16) * count, cudaMemcpyDeviceToDevice, s));
        return RF_OK;
    };
    n->trace_M = n->trace ? M : 0;
    nn::to_bf16(s, n->tdy, n->tdyb, M * nn::C_OUT_P);
    NN_TRY(keep(9, n->tdyb, M * nn::C_OUT_P));
    NN_TRY(wgrad_tc(n, s, 9, n->ta[4], n->tdyb, B, D, H, W));
    NN_TRY(conv(n, s, 9, true, n->tdyb, nullptr, nullptr, n->tgA, B, D, H, W, 0));   // dL/da4
    n->launches += 2;   // mse, to_bf16
    for (int blk = 3; blk >= 0; blk--) {
        nn::relu_bwd(s, n->ta[blk + 1], n->tgA, n->tgB, MH, nullptr);                  // g2
        nn::to_bf16(s, n->tgB, n->tgb, MH);
        NN_TRY(keep(2 + 2 * blk, n->tgb, MH));
        NN_TRY(wgrad_tc(n, s, 2 + 2 * blk, n->tu[blk], n->tgb, B, D, H, W));
        NN_TRY(conv(n, s, 2 + 2 * blk, true, n->tgb, nullptr, nullptr, n->tgA, B, D, H, W, 0));   // du
        nn::relu_bwd(s, n->tu[blk], n->tgA, n->tgC, MH, nullptr);                      // g1
        nn::to_bf16(s, n->tgC, n->tgb, MH);
        NN_TRY(keep(1 + 2 * blk, n->tgb, MH));
        NN_TRY(wgrad_tc(n, s, 1 + 2 * blk, n->ta[blk], n->tgb, B, D, H, W));
        NN_TRY(conv(n, s, 1 + 2 * blk, true, n->tgb, nullptr, nullptr, n->tgA, B, D, H, W, 0));
        nn::add(s, n->tgA, n->tgB, MH);                                                 // + identity branch
        n->launches += 5;   // relu_bwd x2, to_bf16 x2, add
    }
    nn::relu_bwd(s, n->ta[0], n->tgA, n->tgC, MH, nullptr);
    nn::to_bf16(s, n->tgC, n->tgb, MH);
    NN_TRY(keep(0, n->tgb, MH));
    NN_TRY(wgrad_tc(n, s, 0, n->tx, n->tgb, B, D, H, W));
    n->launches += 2;   // relu_bwd, to_bf16
    return RF_OK;
}

rf_status check_dims(int B, int D, int H, int W)
{
    if (B < 1 || D < 1 || H < 1 || W < 1) return nfail(RF_ERR_ARG, "volume dimensions must be positive");
    if ((long long)B * D * H * W > (1LL << 31) / 64) return nfail(RF_ERR_ARG, "volume too large");
    return RF_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Synchronise the network's stream and report a device wait that ran out.
rf_status sync_checked(rf_nn *n)
{
    NN_CUDA(cudaMemcpyAsync(n->fault_h, n->fault, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NN_CUDA(cudaStreamSynchronize(n->stream));
    if (*n->fault_h) return nfail(RF_ERR_DEVICE_TIMEOUT, "warm-start network: a device wait ran out");
    return RF_OK;
}

}  // namespace

// Warm-start guess for a mesh (called by the solver): hk = h + y out_scale dt.
rf_status rf_nn_mesh_guess(rf_nn *n, cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h,
                           const double *Ks, const nn::WsScales &sc, float q_feat, float dt_feat, double scale,
                           double *hk, int *fault)
{
    NN_TRY(ensure_inference(n, g.N));
    NN_TRY(begin(n, s));
    nn::ws_features_bf16(s, g, flags, h, Ks, sc, q_feat, dt_feat, n->ix);
    n->launches++;
    NN_TRY(forward(n, s, n->ix, 1, g.nz, g.ny, g.nx, n->iy, false, fault));
    nn::ws_guess(s, g, flags, h, n->iy, scale, hk);
    n->launches++;
    return end(n, s);
}

extern "C" {

rf_status rf_nn_create(void *cuda_stream, const rf_allocator *alloc, rf_nn **out)
{
    if (!out) return nfail(RF_ERR_ARG, "out is NULL");
    *out = nullptr;
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return nfail(RF_ERR_NO_DEVICE, "no CUDA device");
    NN_CUDA(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    NN_CUDA(cudaGetDeviceProperties(&prop, dev));
    if (prop.major * 10 + prop.minor != 103) return nfail(RF_ERR_NO_DEVICE, "an sm_103 GPU is required");
    rf_nn *n = new rf_nn();
    n->device = dev;
    n->num_sms = prop.multiProcessorCount;
    n->stream = static_cast<cudaStream_t>(cuda_stream);
    if (alloc && alloc->alloc && alloc->free) {
        n->alloc = *alloc;
        n->has_alloc = true;
    }
    layout(n);
    bool ok = cudaEventCreateWithFlags(&n->ev, cudaEventDisableTiming) == cudaSuccess && nalloc(n, n->P, n->nP) &&
              nalloc(n, n->G, n->nP) && nalloc(n, n->M1, n->nP) && nalloc(n, n->M2, n->nP) &&
              nalloc(n, n->Wb, n->nWb) && nalloc(n, n->Wt, n->nWt) && nalloc(n, n->loss_d, 1) &&
              nalloc(n, n->fault, 1) && nalloc(n, n->tcw0, 32 * 27 * 16) && nalloc(n, n->tcw9, 16 * 27 * 32) &&
              nalloc(n, n->tcw9t, 32 * 27 * 16) && cudaMallocHost(&n->loss_h, sizeof(float)) == cudaSuccess &&
              cudaMallocHost(&n->fault_h, sizeof(int)) == cudaSuccess;
    if (ok) {
        cudaStream_t s = n->stream;
        for (void *p : {(void *)n->P, (void *)n->G, (void *)n->M1, (void *)n->M2})
            ok = ok && cudaMemsetAsync(p, 0, sizeof(float) * n->nP, s) == cudaSuccess;
        ok = ok && cudaMemsetAsync(n->fault, 0, sizeof(int), s) == cudaSuccess &&
             cudaMemsetAsync(n->Wb, 0, sizeof(__nv_bfloat16) * n->nWb, s) == cudaSuccess &&
             cudaMemsetAsync(n->Wt, 0, sizeof(__nv_bfloat16) * n->nWt, s) == cudaSuccess &&
             cudaEventRecord(n->ev, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
    }
    if (!ok) {
        rf_nn_destroy(n);
        return nfail(RF_ERR_NOMEM, "warm-start network: allocation failed");
    }
    *out = n;
    return RF_OK;
}

void rf_nn_destroy(rf_nn *n)
{
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    else cudaDeviceSynchronize();
    for (void *p : n->allocations) {
        if (n->has_alloc) n->alloc.free(p, n->alloc.user);
        else cudaFree(p);
    }
    if (n->loss_h) cudaFreeHost(n->loss_h);
    if (n->fault_h) cudaFreeHost(n->fault_h);
    if (n->ev) cudaEventDestroy(n->ev);
    delete n;
}

rf_status rf_nn_set_params(rf_nn *n, const float *params, long long count)
{
    if (!n || !params) return nfail(RF_ERR_ARG, "NULL argument");
    if (count != RF_NN_PARAMS) return nfail(RF_ERR_ARG, "parameter count must be RF_NN_PARAMS");
    std::vector<float> P((size_t)n->nP, 0.0f);
    long long o = 0;
    for (int l = 0; l < nn::N_LAYERS; l++) {
        const LayerDims &d = n->L[l];
        for (int co = 0; co < d.cout; co++)
            for (int tap = 0; tap < 27; tap++)
                for (int ci = 0; ci < d.cin; ci++) {
                    const float v = params[o++];
                    if (!std::isfinite(v)) return nfail(RF_ERR_ARG, "non-finite parameter");
                    P[(size_t)(d.w + (long long)co * d.kp + tap * d.cinp + ci)] = v;
                }
        for (int co = 0; co < d.cout; co++) {
            const float v = params[o++];
            if (!std::isfinite(v)) return nfail(RF_ERR_ARG, "non-finite parameter");
            P[(size_t)(d.b + co)] = v;
        }
    }
    cudaStream_t s = n->stream;
    NN_TRY(begin(n, s));
    NN_CUDA(cudaMemcpyAsync(n->P, P.data(), sizeof(float) * n->nP, cudaMemcpyHostToDevice, s));
    NN_CUDA(cudaMemsetAsync(n->M1, 0, sizeof(float) * n->nP, s));
    NN_CUDA(cudaMemsetAsync(n->M2, 0, sizeof(float) * n->nP, s));
    NN_TRY(refresh_weights(n, s));
    n->adam_t = 0;
    NN_TRY(end(n, s));
    NN_CUDA(cudaStreamSynchronize(s));
    return RF_OK;
}

static rf_status copy_out_logical(rf_nn *n, const float *dev_padded, float *params)
{
    std::vector<float> P((size_t)n->nP);
    NN_CUDA(cudaMemcpyAsync(P.data(), dev_padded, sizeof(float) * n->nP, cudaMemcpyDeviceToHost, n->stream));
    NN_CUDA(cudaStreamSynchronize(n->stream));
    long long o = 0;
    for (int l = 0; l < nn::N_LAYERS; l++) {
        const LayerDims &d = n->L[l];
        for (int co = 0; co < d.cout; co++)
            for (int tap = 0; tap < 27; tap++)
                for (int ci = 0; ci < d.cin; ci++) params[o++] = P[(size_t)(d.w + (long long)co * d.kp + tap * d.cinp + ci)];
        for (int co = 0; co < d.cout; co++) params[o++] = P[(size_t)(d.b + co)];
    }
    return RF_OK;
}

rf_status rf_nn_get_params(rf_nn *n, float *params, long long count)
{
    if (!n || !params) return nfail(RF_ERR_ARG, "NULL argument");
    if (count != RF_NN_PARAMS) return nfail(RF_ERR_ARG, "parameter count must be RF_NN_PARAMS");
    NN_TRY(begin(n, n->stream));
    return copy_out_logical(n, n->P, params);
}

rf_status rf_nn_forward(rf_nn *n, const float *d_x, int B, int D, int H, int W, float *d_y)
{
    rf::NvtxRange range("rf_nn_forward");
    if (!n || !d_x || !d_y) return nfail(RF_ERR_ARG, "NULL argument");
    if (!aligned16(d_x)) return nfail(RF_ERR_ARG, "d_x must be 16-byte aligned");
    NN_TRY(check_dims(B, D, H, W));
    const long long M = (long long)B * D * H * W;
    NN_TRY(ensure_inference(n, M));
    cudaStream_t s = n->stream;
    NN_TRY(begin(n, s));
    nn::pad_features(s, d_x, n->ix, M);
    n->launches++;
    NN_TRY(forward(n, s, n->ix, B, D, H, W, n->iy, false));
    k_take0<<<(int)std::min<long long>((M + 255) / 256, 4096), 256, 0, s>>>(n->iy, d_y, M);
    n->launches++;
    return end(n, s);
}

rf_status rf_nn_loss_grad(rf_nn *n, const float *d_x, const float *d_target, const float *d_mask, int B, int D,
                          int H, int W, float *loss, float *grad)
{
    rf::NvtxRange range("rf_nn_loss_grad");
    if (!n || !d_x || !d_target) return nfail(RF_ERR_ARG, "NULL argument");
    if (!aligned16(d_x)) return nfail(RF_ERR_ARG, "d_x must be 16-byte aligned");
    NN_TRY(check_dims(B, D, H, W));
    NN_TRY(begin(n, n->stream));
    NN_TRY(loss_grad(n, d_x, d_target, d_mask, B, D, H, W));
    NN_CUDA(cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NN_TRY(end(n, n->stream));
    if (grad) NN_TRY(copy_out_logical(n, n->G, grad));
    NN_TRY(sync_checked(n));
    if (loss) *loss = *n->loss_h;
    return RF_OK;
}

rf_status rf_nn_train_step(rf_nn *n, const float *d_x, const float *d_target, const float *d_mask, int B, int D,
                           int H, int W, const rf_adam *opt, float *loss)
{
    rf::NvtxRange range("rf_nn_train_step");
    if (!n || !d_x || !d_target || !opt) return nfail(RF_ERR_ARG, "NULL argument");
    if (!aligned16(d_x)) return nfail(RF_ERR_ARG, "d_x must be 16-byte aligned");
    if (!(opt->lr > 0) || !(opt->beta1 >= 0 && opt->beta1 < 1) || !(opt->beta2 >= 0 && opt->beta2 < 1) ||
        !(opt->eps > 0))
        return nfail(RF_ERR_ARG, "invalid Adam settings");
    NN_TRY(check_dims(B, D, H, W));
    cudaStream_t s = n->stream;
    NN_TRY(begin(n, s));
    NN_TRY(loss_grad(n, d_x, d_target, d_mask, B, D, H, W));
    n->adam_t++;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)opt->beta1, n->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)opt->beta2, n->adam_t)));
    nn::adam(s, n->P, n->G, n->M1, n->M2, n->nP, opt->lr, opt->beta1, opt->beta2, opt->eps, c1, c2);
    n->launches++;
    NN_TRY(refresh_weights(n, s));
    if (loss) NN_CUDA(cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(float), cudaMemcpyDeviceToHost, s));
    NN_TRY(end(n, s));
    if (loss) {
        NN_TRY(sync_checked(n));
        *loss = *n->loss_h;
    }
    return RF_OK;
}

long long rf_nn_launch_count(const rf_nn *n) { return n ? n->launches : 0; }

rf_status rf_nn_set_trace(rf_nn *n, int on)
{
    if (!n) return nfail(RF_ERR_ARG, "NULL argument");
    n->trace = on != 0;
    n->trace_M = 0;
    return RF_OK;
}

rf_status rf_nn_trace_get(rf_nn *n, int what, int index, void *host, long long count)
{
    if (!n || !host) return nfail(RF_ERR_ARG, "NULL argument");
    const long long M = n->trace_M;
    if (M < 1) return nfail(RF_ERR_STATE, "no traced gradient evaluation (rf_nn_set_trace, then rf_nn_loss_grad)");
    const void *src = nullptr;
    long long expect = 0;
    size_t elem = sizeof(__nv_bfloat16);
    switch (what) {
    case RF_NN_TRACE_INPUT:
        if (index != 0) break;
        src = n->tx, expect = M * nn::C_IN_P;
        break;
    case RF_NN_TRACE_BLOCK_OUT:
        if (index < 0 || index > 4) break;
        src = n->ta[index], expect = M * nn::C_HID;
        break;
    case RF_NN_TRACE_BLOCK_MID:
        if (index < 0 || index > 3) break;
        src = n->tu[index], expect = M * nn::C_HID;
        break;
    case RF_NN_TRACE_OUT_GRAD:
        if (index < 0 || index >= nn::N_LAYERS) break;
        src = n->trace_g[index], expect = M * (index == nn::N_LAYERS - 1 ? nn::C_OUT_P : nn::C_HID);
        break;
    case RF_NN_TRACE_OUTPUT:
        if (index != 0) break;
        src = n->ty, expect = M * nn::C_OUT_P, elem = sizeof(float);
        break;
    default:
        break;
    }
    if (!src) return nfail(RF_ERR_ARG, "rf_nn_trace_get: unknown tensor or index");
    if (count != expect) return nfail(RF_ERR_ARG, "rf_nn_trace_get: count does not match the tensor's size");
    NN_CUDA(cudaStreamSynchronize(n->stream));
    NN_CUDA(cudaMemcpy(host, src, elem * (size_t)count, cudaMemcpyDeviceToHost));
    return RF_OK;
}

}  // extern "C"
