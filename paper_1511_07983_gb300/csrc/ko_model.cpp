// Surrogate model: parameters, training on simulator-labelled orders, and
// proposal of orders for sets too large to enumerate, every proposal rescored
// exactly by the run-length simulator.  (The paper has no learned component;
// this serves the same goal as Algorithm 1 -- a good launch order without
// trying all N! -- and every result it returns is an exactly simulated makespan.)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ko_fast.h"
#include "ko_mlp.h"

namespace {

constexpr double kBeta1 = 0.9, kBeta2 = 0.999, kEps = 1e-8;

template <typename T>
bool dalloc(T **p, size_t n)
{
    if (cudaMalloc((void **)p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// standard normal from two SplitMix64 draws (Box-Muller)
double normal(uint64_t seed, uint64_t i)
{
    const double u1 = ((mix64(seed + (2 * i + 1) * 0x9E3779B97F4A7C15ull) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (mix64(seed + (2 * i + 2) * 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

// Per-set descriptors the encoder reads: kernel features [24][7], globals [8].
void ko_set_features(const KoSet &h, int64_t lb, float *kf, float *gf)
{
    std::memset(kf, 0, sizeof(float) * kMaxK * kSlotFeat);
    for (int i = 0; i < h.n; i++) {
        const KoKern &k = h.k[i];
        float *f = kf + i * kSlotFeat;
        f[0] = (float)((double)k.r / (double)h.R);
        f[1] = (float)((double)k.s / (double)h.Sh);
        f[2] = (float)((double)k.w / (double)h.W);
        f[3] = (float)((double)((k.b + h.S - 1) / h.S) / (double)h.Bk);
        f[4] = (float)(std::log2((double)k.c) / 16.0);
        f[5] = (float)(std::log2((double)k.m) / 16.0);
        f[6] = 1.0f;
    }
    gf[0] = (float)(h.n / 24.0);
    gf[1] = (float)(h.S / 148.0);
    gf[2] = (float)(std::log2((double)h.R) / 24.0);
    gf[3] = (float)(std::log2((double)h.Sh) / 24.0);
    gf[4] = (float)(std::log2((double)h.W) / 24.0);
    gf[5] = (float)(std::log2((double)h.Bk) / 24.0);
    gf[6] = (float)(std::log2((double)(lb > 1 ? lb : 1)) / 32.0);
    gf[7] = 1.0f;
}

struct ko_model {
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    uint16_t *w1t = nullptr, *w2 = nullptr, *w2t = nullptr, *w3 = nullptr, *w3t = nullptr, *w4b = nullptr;
    long long step = 0;
    int cap = 0;  // batch capacity of the activation buffers
    uint16_t *a0 = nullptr, *a0t = nullptr, *a1 = nullptr, *a1t = nullptr, *a2 = nullptr, *a2t = nullptr,
             *a3 = nullptr, *dz = nullptr, *dzt = nullptr;
    float *y = nullptr, *t = nullptr, *da = nullptr, *loss = nullptr;
    float *part = nullptr;     // per-block bias-gradient partials (summed in a fixed order)
    int *pick = nullptr;
    KoFastState fast{};
    int tc_forward = 1;        // inference layers on tcgen05 (1) or mma.sync (0)
    int tc_train = 1;          // training GEMMs on tcgen05 (1) or mma.sync (0)
    float *wg_work = nullptr;  // split-K partials of the tcgen05 weight gradients
    size_t wg_bytes = 0;
    int chunk = 262144;        // candidate rows per forward pass of the proposal paths
    int *tc_err = nullptr;     // device flag: a tcgen05 completion wait gave up
    int polish = 64;           // exact descent steps after a guided search (0: none)

    void free_acts()
    {
        cudaFree(a0); cudaFree(a0t); cudaFree(a1); cudaFree(a1t); cudaFree(a2); cudaFree(a2t); cudaFree(a3);
        cudaFree(dz); cudaFree(dzt); cudaFree(y); cudaFree(t); cudaFree(da); cudaFree(pick); cudaFree(part);
        a0 = a0t = a1 = a1t = a2 = a2t = a3 = dz = dzt = nullptr;
        y = t = da = part = nullptr;
        pick = nullptr;
        cap = 0;
    }
    ~ko_model()
    {
        free_acts();
        cudaFree(p); cudaFree(m); cudaFree(v); cudaFree(g); cudaFree(loss); cudaFree(tc_err); cudaFree(wg_work);
        cudaFree(w1t); cudaFree(w2); cudaFree(w2t); cudaFree(w3); cudaFree(w3t); cudaFree(w4b);
        ko_fast_release(&fast);
    }
};

namespace {

ko_status ensure_acts(ko_model *md, int B)
{
    if (md->cap >= B) return KO_OK;
    md->free_acts();
    const size_t in = (size_t)B * kMlpIn, hid = (size_t)B * kHidden;
    bool ok = dalloc(&md->a0, in) && dalloc(&md->a0t, in) && dalloc(&md->a1, hid) && dalloc(&md->a1t, hid) &&
              dalloc(&md->a2, hid) && dalloc(&md->a2t, hid) && dalloc(&md->a3, hid) && dalloc(&md->dz, hid) &&
              dalloc(&md->dzt, hid) && dalloc(&md->y, (size_t)B) && dalloc(&md->t, (size_t)B) &&
              dalloc(&md->da, hid) && dalloc(&md->pick, (size_t)B) && dalloc(&md->part, ko_mlp_part_floats(B));
    if (!ok) {
        md->free_acts();
        return KO_ERR_NOMEM;
    }
    md->cap = B;
    return KO_OK;
}

ko_status cuda_ok(cudaError_t e)
{
    if (e == cudaSuccess) return KO_OK;
    cudaGetLastError();
    return KO_ERR_CUDA;
}

// Two timing events; both null on failure.
static ko_status make_events(cudaEvent_t *e0, cudaEvent_t *e1)
{
    if (cudaEventCreate(e0) != cudaSuccess || cudaEventCreate(e1) != cudaSuccess) {
        cudaGetLastError();
        if (*e0) cudaEventDestroy(*e0);
        *e0 = *e1 = nullptr;
        return KO_ERR_CUDA;
    }
    return KO_OK;
}

ko_status refresh_bf16(ko_model *md, cudaStream_t st)
{
    ko_status s;
    if ((s = cuda_ok(ko_mlp_weights_bf16(md->p + kOffW1, kMlpIn, kHidden, nullptr, md->w1t, st)))) return s;
    if ((s = cuda_ok(ko_mlp_weights_bf16(md->p + kOffW2, kHidden, kHidden, md->w2, md->w2t, st)))) return s;
    if ((s = cuda_ok(ko_mlp_weights_bf16(md->p + kOffW3, kHidden, kHidden, md->w3, md->w3t, st)))) return s;
    return cuda_ok(ko_mlp_weights_bf16(md->p + kOffW4, kHidden, 1, md->w4b, nullptr, st));
}

// Forward over a0 (B rows, B % 64 == 0); with `train` the transposed
// activations for the weight gradients are written too.
ko_status forward(ko_model *md, int B, bool train, cudaStream_t st)
{
    ko_status s;
    if (train && md->tc_train && B % 128 == 0) {
        // a layer the tcgen05 path cannot take (shared memory) is refused before launch: use mma.sync
        const cudaError_t e = ko_mlp_layer_tc_t(md->a0, md->w1t, B, kMlpIn, md->p + kOffB1, md->a1, md->a1t, B,
                                                md->tc_err, st);
        if (e == cudaSuccess) {
            if ((s = cuda_ok(ko_mlp_layer_tc_t(md->a1, md->w2t, B, kHidden, md->p + kOffB2, md->a2, md->a2t, B,
                                               md->tc_err, st))))
                return s;
            if ((s = cuda_ok(ko_mlp_layer_tc(md->a2, md->w3t, B, kHidden, md->p + kOffB3, md->a3, md->tc_err, st))))
                return s;
            return cuda_ok(ko_mlp_out_fwd(md->a3, md->w4b, md->p + kOffB4, B, md->y, st));
        }
        if (e != cudaErrorInvalidValue) return cuda_ok(e);
        cudaGetLastError();
        md->tc_train = 0;
    }
    if (!train && md->tc_forward && B % 128 == 0) {
        if ((s = cuda_ok(ko_mlp_layer_tc(md->a0, md->w1t, B, kMlpIn, md->p + kOffB1, md->a1, md->tc_err, st)))) return s;
        if ((s = cuda_ok(ko_mlp_layer_tc(md->a1, md->w2t, B, kHidden, md->p + kOffB2, md->a2, md->tc_err, st)))) return s;
        // the last hidden layer and the output layer in one kernel: a3 is not written
        return cuda_ok(ko_mlp_layer_tc_out(md->a2, md->w3t, B, kHidden, md->p + kOffB3, md->w4b, md->p + kOffB4,
                                           md->a3, md->y, md->tc_err, st));
    }
    if ((s = cuda_ok(ko_mlp_gemm_relu(md->a0, kMlpIn, md->w1t, kMlpIn, B, kHidden, kMlpIn, md->p + kOffB1,
                                      md->a1, kHidden, train ? md->a1t : nullptr, B, st))))
        return s;
    if ((s = cuda_ok(ko_mlp_gemm_relu(md->a1, kHidden, md->w2t, kHidden, B, kHidden, kHidden, md->p + kOffB2,
                                      md->a2, kHidden, train ? md->a2t : nullptr, B, st))))
        return s;
    if ((s = cuda_ok(ko_mlp_gemm_relu(md->a2, kHidden, md->w3t, kHidden, B, kHidden, kHidden, md->p + kOffB3,
                                      md->a3, kHidden, nullptr, 0, st))))
        return s;
    return cuda_ok(ko_mlp_out_fwd(md->a3, md->w4b, md->p + kOffB4, B, md->y, st));
}

// Gradients of the mean squared error into md->g (zeroed here); loss sum
// added to *loss_dev.
// tcgen05 weight and input gradients (B % 256 == 0), the mma.sync ones otherwise.
ko_status wgrad(ko_model *md, const uint16_t *at, int M, int B, float *out, cudaStream_t st)
{
    if (md->tc_train && B % 256 == 0) {
        const size_t need = ko_mlp_wgrad_tc_workspace(M, B);
        if (md->wg_bytes < need) {
            cudaFree(md->wg_work);
            md->wg_work = nullptr;
            md->wg_bytes = 0;
            if (cudaMalloc(&md->wg_work, need) != cudaSuccess) {
                cudaGetLastError();
                return KO_ERR_NOMEM;
            }
            md->wg_bytes = need;
        }
        const cudaError_t e = ko_mlp_wgrad_tc(at, B, md->dzt, B, M, B, out, kHidden, md->wg_work, md->tc_err, st);
        if (e != cudaErrorInvalidValue) return cuda_ok(e);
        cudaGetLastError();
    }
    return cuda_ok(ko_mlp_gemm_f32(at, B, md->dzt, B, M, kHidden, B, out, kHidden, st));
}

ko_status dgrad(ko_model *md, const uint16_t *w, int B, cudaStream_t st)
{
    if (md->tc_train && B % 128 == 0) {
        const cudaError_t e = ko_mlp_layer_tc_f32(md->dz, w, B, kHidden, md->da, md->tc_err, st);
        if (e != cudaErrorInvalidValue) return cuda_ok(e);
        cudaGetLastError();
    }
    return cuda_ok(ko_mlp_gemm_f32(md->dz, kHidden, w, kHidden, B, kHidden, kHidden, md->da, kHidden, st));
}

ko_status backward(ko_model *md, int B, float *loss_dev, cudaStream_t st)
{
    ko_status s;
    if (cudaMemsetAsync(md->g, 0, sizeof(float) * kParams, st) != cudaSuccess) return KO_ERR_CUDA;
    if ((s = cuda_ok(ko_mlp_out_bwd(md->y, md->t, md->a3, md->w4b, B, loss_dev, md->g + kOffW4, md->g + kOffB4,
                                    md->g + kOffB3, md->dz, md->dzt, md->part, st))))
        return s;
    if (md->tc_train) {
        if ((s = wgrad(md, md->a2t, kHidden, B, md->g + kOffW3, st))) return s;
        if ((s = dgrad(md, md->w3, B, st))) return s;
        if ((s = cuda_ok(ko_mlp_relu_bwd(md->da, md->a2, B, md->g + kOffB2, md->dz, md->dzt, md->part, st)))) return s;
        if ((s = wgrad(md, md->a1t, kHidden, B, md->g + kOffW2, st))) return s;
        if ((s = dgrad(md, md->w2, B, st))) return s;
        if ((s = cuda_ok(ko_mlp_relu_bwd(md->da, md->a1, B, md->g + kOffB1, md->dz, md->dzt, md->part, st)))) return s;
        return wgrad(md, md->a0t, kMlpIn, B, md->g + kOffW1, st);
    }
    // layer 3
    if ((s = cuda_ok(ko_mlp_gemm_f32(md->a2t, B, md->dzt, B, kHidden, kHidden, B, md->g + kOffW3, kHidden, st))))
        return s;
    if ((s = cuda_ok(ko_mlp_gemm_f32(md->dz, kHidden, md->w3, kHidden, B, kHidden, kHidden, md->da, kHidden, st))))
        return s;
    if ((s = cuda_ok(ko_mlp_relu_bwd(md->da, md->a2, B, md->g + kOffB2, md->dz, md->dzt, md->part, st)))) return s;
    // layer 2
    if ((s = cuda_ok(ko_mlp_gemm_f32(md->a1t, B, md->dzt, B, kHidden, kHidden, B, md->g + kOffW2, kHidden, st))))
        return s;
    if ((s = cuda_ok(ko_mlp_gemm_f32(md->dz, kHidden, md->w2, kHidden, B, kHidden, kHidden, md->da, kHidden, st))))
        return s;
    if ((s = cuda_ok(ko_mlp_relu_bwd(md->da, md->a1, B, md->g + kOffB1, md->dz, md->dzt, md->part, st)))) return s;
    // layer 1 (no input gradient needed)
    return cuda_ok(ko_mlp_gemm_f32(md->a0t, B, md->dzt, B, kMlpIn, kHidden, B, md->g + kOffW1, kHidden, st));
}

ko_status adam(ko_model *md, float lr, cudaStream_t st)
{
    md->step++;
    const float c1 = (float)(1.0 - std::pow(kBeta1, (double)md->step));
    const float c2 = (float)(1.0 - std::pow(kBeta2, (double)md->step));
    ko_status s = cuda_ok(ko_mlp_adam(md->p, md->m, md->v, md->g, kParams, lr, (float)kBeta1, (float)kBeta2,
                                      (float)kEps, c1, c2, st));
    if (s) return s;
    return refresh_bf16(md, st);
}

uint16_t host_bf16(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Features of raw rows x [B x 192] (host floats) into a0 / a0t.
ko_status upload_features(ko_model *md, const float *x, int B, cudaStream_t st)
{
    std::vector<uint16_t> h((size_t)B * kMlpIn), ht((size_t)B * kMlpIn);
    for (int b = 0; b < B; b++)
        for (int f = 0; f < kMlpIn; f++) {
            const uint16_t v = host_bf16(x[(size_t)b * kMlpIn + f]);
            h[(size_t)b * kMlpIn + f] = v;
            ht[(size_t)f * B + b] = v;
        }
    if (cudaMemcpyAsync(md->a0, h.data(), h.size() * 2, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(md->a0t, ht.data(), ht.size() * 2, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return KO_ERR_CUDA;
    return KO_OK;
}

}  // namespace

// ---------------------------------------------------------------------- ABI
ko_model *ko_model_new(uint64_t seed, ko_status *err)
{
    ko_model *md = new (std::nothrow) ko_model();
    if (!md) { *err = KO_ERR_NOMEM; return nullptr; }
    bool ok = dalloc(&md->p, kParams) && dalloc(&md->m, kParams) && dalloc(&md->v, kParams) &&
              dalloc(&md->g, kParams) && dalloc(&md->w1t, (size_t)kMlpIn * kHidden) &&
              dalloc(&md->w2, (size_t)kHidden * kHidden) && dalloc(&md->w2t, (size_t)kHidden * kHidden) &&
              dalloc(&md->w3, (size_t)kHidden * kHidden) && dalloc(&md->w3t, (size_t)kHidden * kHidden) &&
              dalloc(&md->w4b, (size_t)kHidden) && dalloc(&md->loss, 1 << 16) && dalloc(&md->tc_err, 1);
    if (!ok) { delete md; *err = KO_ERR_NOMEM; return nullptr; }
    // He-normal initialisation from a counter-based generator (zero biases,
    // zero weights on the padded input features)
    std::vector<float> h(kParams, 0.0f);
    uint64_t ctr = 0;
    for (int k = 0; k < kMlpIn; k++)
        for (int n = 0; n < kHidden; n++, ctr++)
            h[kOffW1 + (long long)k * kHidden + n] =
                k < kSlots * kSlotFeat + kGlobals ? (float)(normal(seed, ctr) * std::sqrt(2.0 / 176.0)) : 0.0f;
    for (long long i = 0; i < (long long)kHidden * kHidden; i++, ctr++) h[kOffW2 + i] = (float)(normal(seed, ctr) * std::sqrt(2.0 / kHidden));
    for (long long i = 0; i < (long long)kHidden * kHidden; i++, ctr++) h[kOffW3 + i] = (float)(normal(seed, ctr) * std::sqrt(2.0 / kHidden));
    for (int i = 0; i < kHidden; i++, ctr++) h[kOffW4 + i] = (float)(normal(seed, ctr) * std::sqrt(1.0 / kHidden));
    *err = ko_model_load(md, h.data());
    if (*err) { delete md; return nullptr; }
    return md;
}

ko_status ko_model_load(ko_model *md, const float *params)
{
    if (cudaMemcpy(md->p, params, sizeof(float) * kParams, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(md->m, 0, sizeof(float) * kParams) != cudaSuccess ||
        cudaMemset(md->v, 0, sizeof(float) * kParams) != cudaSuccess)
        return KO_ERR_CUDA;
    md->step = 0;
    ko_status s = refresh_bf16(md, nullptr);
    if (s) return s;
    return cudaDeviceSynchronize() == cudaSuccess ? KO_OK : KO_ERR_CUDA;
}

ko_status ko_model_store(const ko_model *md, float *params)
{
    return cudaMemcpy(params, md->p, sizeof(float) * kParams, cudaMemcpyDeviceToHost) == cudaSuccess ? KO_OK
                                                                                                      : KO_ERR_CUDA;
}

void ko_model_free(ko_model *md) { delete md; }

ko_status ko_model_option(ko_model *md, int key, long long value)
{
    if (key == KO_MODEL_OPT_TC) {
        if (value != 0 && value != 1) return KO_ERR_ARG;
        md->tc_forward = (int)value;
        if (cudaMemset(md->tc_err, 0, sizeof(int)) != cudaSuccess) return KO_ERR_CUDA;
        return KO_OK;
    }
    if (key == KO_MODEL_OPT_TC_TRAIN) {
        if (value != 0 && value != 1) return KO_ERR_ARG;
        md->tc_train = (int)value;
        if (cudaMemset(md->tc_err, 0, sizeof(int)) != cudaSuccess) return KO_ERR_CUDA;
        return KO_OK;
    }
    if (key == KO_MODEL_OPT_CHUNK) {
        if (value < 1024 || value > (1 << 22) || value % 1024) return KO_ERR_ARG;
        md->chunk = (int)value;
        return KO_OK;
    }
    if (key == KO_MODEL_OPT_POLISH) {
        if (value < 0 || value > (1 << 20)) return KO_ERR_ARG;
        md->polish = (int)value;
        return KO_OK;
    }
    return KO_ERR_ARG;
}

// KO_ERR_TIMEOUT if a tcgen05 layer reported that its completion wait gave up.
ko_status ko_model_check(ko_model *md)
{
    int e = 0;
    if (cudaMemcpy(&e, md->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return KO_ERR_CUDA;
    return e ? KO_ERR_TIMEOUT : KO_OK;
}

// Raw features: forward, and optionally backward (+ Adam when lr > 0).
ko_status ko_model_raw(ko_model *md, const float *x, const float *t, int B, float *y_out, float *grad_out,
                       float *loss_out, float lr, cudaStream_t st)
{
    if (B < 64 || B % 64) return KO_ERR_ARG;
    ko_status s = ensure_acts(md, B);
    if (s) return s;
    if ((s = upload_features(md, x, B, st))) return s;
    if ((s = forward(md, B, t != nullptr, st))) return s;
    if (t) {
        if (cudaMemcpyAsync(md->t, t, sizeof(float) * B, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(md->loss, 0, sizeof(float), st) != cudaSuccess)
            return KO_ERR_CUDA;
        if ((s = backward(md, B, md->loss, st))) return s;
        if (grad_out && cudaMemcpyAsync(grad_out, md->g, sizeof(float) * kParams, cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess)
            return KO_ERR_CUDA;
        if (lr > 0.0f && (s = adam(md, lr, st))) return s;
        float ls = 0.0f;
        if (cudaMemcpyAsync(&ls, md->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return KO_ERR_CUDA;
        if (loss_out) *loss_out = ls / (float)B;
    }
    if (y_out && cudaMemcpyAsync(y_out, md->y, sizeof(float) * B, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return KO_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return KO_ERR_CUDA;
    return ko_model_check(md);
}

// ------------------------------------------------------------ set plumbing

struct SetTables {
    int *set_n = nullptr;
    float *kfeat = nullptr, *gfeat = nullptr;
    double *log2_lb = nullptr;
    KoSet *sets = nullptr;
    ~SetTables()
    {
        cudaFree(set_n); cudaFree(kfeat); cudaFree(gfeat); cudaFree(log2_lb); cudaFree(sets);
    }
};

static ko_status build_tables(const KoSet *const *hs, int nsets, SetTables *tb, cudaStream_t st)
{
    std::vector<int> n(nsets);
    std::vector<float> kf((size_t)nsets * kMaxK * kSlotFeat), gf((size_t)nsets * kGlobals);
    std::vector<double> l2(nsets);
    std::vector<KoSet> sets(nsets);
    for (int i = 0; i < nsets; i++) {
        int64_t lb = 0, ub = 0;
        ko_bounds_host(*hs[i], &lb, &ub);
        n[i] = hs[i]->n;
        ko_set_features(*hs[i], lb, kf.data() + (size_t)i * kMaxK * kSlotFeat, gf.data() + (size_t)i * kGlobals);
        l2[i] = std::log2((double)(lb > 1 ? lb : 1));
        sets[i] = *hs[i];
        sets[i].ref_makespan = 0;
    }
    if (!dalloc(&tb->set_n, nsets) || !dalloc(&tb->kfeat, kf.size()) || !dalloc(&tb->gfeat, gf.size()) ||
        !dalloc(&tb->log2_lb, nsets) || !dalloc(&tb->sets, nsets))
        return KO_ERR_NOMEM;
    if (cudaMemcpyAsync(tb->set_n, n.data(), sizeof(int) * nsets, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(tb->kfeat, kf.data(), sizeof(float) * kf.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(tb->gfeat, gf.data(), sizeof(float) * gf.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(tb->log2_lb, l2.data(), sizeof(double) * nsets, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(tb->sets, sets.data(), sizeof(KoSet) * nsets, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return KO_ERR_CUDA;
    return KO_OK;
}

// Threads per simulation for `count` explicit orders of set h (measured on a
// GB300 with 16- to 24-kernel sets): with more than 32 SMs the runs of
// distinct SM states outgrow 16 lanes and the one-thread state, so 32 lanes;
// otherwise 32 lanes up to 4096 orders (the latency of single simulations
// decides), 16 up to 32768, one thread per order beyond.
static int row_lanes(const KoSet &h, long long count)
{
    if (h.S > 32 || count <= 4096) return 32;
    return count <= 32768 ? 16 : 1;
}

// Exact makespans of `count` rows (stride 24) of set `set` into out, with the
// threads per simulation of row_lanes (the state's own choice is kept).
static ko_status exact_rows(KoFastState *fs, const KoSet *d_sets, const KoSet &h, int set, const int8_t *rows,
                            long long count, int64_t *out, KoChunk *d_chunk, cudaStream_t st)
{
    struct Keep {  // restores the state's lanes and state size on every return
        KoFastState *fs;
        int lanes, shape;
        ~Keep() { fs->lanes = lanes; fs->lane_shape = shape; }
    } keep{fs, fs->lanes, fs->lane_shape};
    fs->lanes = row_lanes(h, count);
    fs->lane_shape = 0;
    KoChunk c{};
    c.count = count;
    c.set = set;
    c.d0 = h.n;
    c.mode = 2;
    if (cudaMemcpyAsync(d_chunk, &c, sizeof(c), cudaMemcpyHostToDevice, st) != cudaSuccess) return KO_ERR_CUDA;
    KoWork w{};
    w.sets = d_sets;
    w.chunks = d_chunk;
    w.nchunks = 1;
    w.n_items = count;
    w.perms = rows;
    w.perm_stride = kMaxK;
    w.out = out;
    w.levels = 1;
    return ko_fast_launch(fs, w, ko_slab_bytes(h.S, h.Bk), st);
}

ko_status ko_model_train_sets(ko_model *md, const KoSet *const *hs, int nsets, long long pairs_per_set,
                              int steps, int batch, float lr, uint64_t seed, float *loss_curve, cudaStream_t st)
{
    if (nsets < 1 || pairs_per_set < 1 || steps < 1 || batch < 64 || batch % 64 || steps > (1 << 16))
        return KO_ERR_ARG;
    for (int i = 0; i < nsets; i++)
        if (!ko_fast_applicable(*hs[i])) return KO_ERR_OVERFLOW;
    SetTables tb;
    ko_status s = build_tables(hs, nsets, &tb, st);
    if (s) return s;
    const long long pool = (long long)nsets * pairs_per_set;
    int8_t *rows = nullptr;
    int64_t *ms = nullptr;
    float *targets = nullptr;
    int *sid = nullptr;
    KoChunk *d_chunk = nullptr;
    if (!dalloc(&rows, (size_t)pool * kMaxK) || !dalloc(&ms, (size_t)pool) || !dalloc(&targets, (size_t)pool) ||
        !dalloc(&sid, (size_t)pool) || !dalloc(&d_chunk, 1)) {
        cudaFree(rows); cudaFree(ms); cudaFree(targets); cudaFree(sid); cudaFree(d_chunk);
        return KO_ERR_NOMEM;
    }
    std::vector<int> h_sid(pool);
    for (long long i = 0; i < pool; i++) h_sid[i] = (int)(i / pairs_per_set);
    do {
        if (cudaMemcpyAsync(sid, h_sid.data(), sizeof(int) * pool, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(rows, 0, (size_t)pool * kMaxK, st) != cudaSuccess) { s = KO_ERR_CUDA; break; }
        // labelled pool: uniform random orders of each set, exact makespans, targets
        for (int i = 0; i < nsets && !s; i++) {
            int8_t *r = rows + (size_t)i * pairs_per_set * kMaxK;
            if ((s = cuda_ok(ko_mlp_random_orders(r, kMaxK, pairs_per_set, hs[i]->n, mix64(seed ^ (0x5151ull + i)), st))))
                break;
            s = exact_rows(&md->fast, tb.sets, *hs[i], i, r, pairs_per_set, ms + (size_t)i * pairs_per_set, d_chunk, st);
        }
        if (s) break;
        if ((s = cuda_ok(ko_mlp_targets(ms, sid, tb.log2_lb, pool, targets, st)))) break;
        if ((s = ensure_acts(md, batch))) break;
        if (cudaMemsetAsync(md->loss, 0, sizeof(float) * steps, st) != cudaSuccess) { s = KO_ERR_CUDA; break; }
        for (int it = 0; it < steps && !s; it++) {
            if ((s = cuda_ok(ko_mlp_pick(md->pick, batch, pool, mix64(seed + 0x1000ull + it), targets, md->t, st))))
                break;
            if ((s = cuda_ok(ko_mlp_encode(rows, kMaxK, sid, md->pick, tb.set_n, tb.kfeat, tb.gfeat, batch, md->a0,
                                           md->a0t, st))))
                break;
            if ((s = forward(md, batch, true, st))) break;
            if ((s = backward(md, batch, md->loss + it, st))) break;
            s = adam(md, lr, st);
        }
        if (s) break;
        if (loss_curve) {
            std::vector<float> lc(steps);
            if (cudaMemcpyAsync(lc.data(), md->loss, sizeof(float) * steps, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { s = KO_ERR_CUDA; break; }
            for (int i = 0; i < steps; i++) loss_curve[i] = lc[i] / (float)batch;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) s = KO_ERR_CUDA;
        if (!s) s = ko_model_check(md);  // a tcgen05 completion wait that gave up
    } while (false);
    cudaFree(rows); cudaFree(ms); cudaFree(targets); cudaFree(sid); cudaFree(d_chunk);
    return s;
}

// Best exact makespan among the rows [count x 24] of one set (device), index too.
static ko_status best_of(const int64_t *d_ms, long long count, int64_t *best, long long *best_idx)
{
    std::vector<int64_t> h(count);
    if (cudaMemcpy(h.data(), d_ms, sizeof(int64_t) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
        return KO_ERR_CUDA;
    long long bi = -1;
    for (long long i = 0; i < count; i++)
        if (h[i] >= 0 && (bi < 0 || h[i] < h[bi])) bi = i;
    if (bi < 0) return KO_ERR_STATE;
    *best = h[bi];
    *best_idx = bi;
    return KO_OK;
}

ko_status ko_model_propose_set(ko_model *md, const KoSet &h, long long n_cand, int top_k, uint64_t seed,
                               int32_t *best_order, int64_t *best_makespan, double *gpu_ms, cudaStream_t st)
{
    if (n_cand < 1 || top_k < 1 || top_k > n_cand || n_cand > (1ll << 26)) return KO_ERR_ARG;
    if (!ko_fast_applicable(h)) return KO_ERR_OVERFLOW;
    const KoSet *hs[1] = {&h};
    SetTables tb;
    ko_status s = build_tables(hs, 1, &tb, st);
    if (s) return s;
    const int C = md->chunk;
    const long long padded = (n_cand + C - 1) / C * C;
    int8_t *rows = nullptr, *top_rows = nullptr;
    float *y_all = nullptr;
    int *top_idx = nullptr;
    int64_t *top_ms = nullptr;
    uint32_t *sel_state = nullptr;
    unsigned int *sel_hist = nullptr, *sel_cnt = nullptr;
    KoChunk *d_chunk = nullptr;
    if (!dalloc(&rows, (size_t)padded * kMaxK) || !dalloc(&y_all, (size_t)n_cand) || !dalloc(&top_idx, top_k) ||
        !dalloc(&top_rows, (size_t)top_k * kMaxK) || !dalloc(&top_ms, top_k) || !dalloc(&sel_state, 2) ||
        !dalloc(&sel_hist, 256) || !dalloc(&sel_cnt, 2) || !dalloc(&d_chunk, 1)) {
        s = KO_ERR_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!s) s = make_events(&e0, &e1);
    if (!s) s = ensure_acts(md, C);
    if (!s) {
        cudaEventRecord(e0, st);
        if (cudaMemsetAsync(rows, 0, (size_t)padded * kMaxK, st) != cudaSuccess) s = KO_ERR_CUDA;
        if (!s) s = cuda_ok(ko_mlp_random_orders(rows, kMaxK, n_cand, h.n, mix64(seed ^ 0xC0FFEEull), st));
        for (long long off = 0; off < n_cand && !s; off += C) {
            const long long c = n_cand - off < C ? n_cand - off : C;
            if ((s = cuda_ok(ko_mlp_encode(rows + (size_t)off * kMaxK, kMaxK, nullptr, nullptr, tb.set_n, tb.kfeat,
                                           tb.gfeat, C, md->a0, nullptr, st))))
                break;
            if ((s = forward(md, C, false, st))) break;
            if (cudaMemcpyAsync(y_all + off, md->y, sizeof(float) * c, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                s = KO_ERR_CUDA;
        }
        if (!s) s = cuda_ok(ko_mlp_topk(y_all, n_cand, top_k, sel_state, sel_hist, sel_cnt, top_idx, st));
        if (!s) s = cuda_ok(ko_mlp_gather_rows(rows, kMaxK, top_idx, top_k, top_rows, st));
        if (!s) s = exact_rows(&md->fast, tb.sets, h, 0, top_rows, top_k, top_ms, d_chunk, st);
        cudaEventRecord(e1, st);
        if (!s && cudaStreamSynchronize(st) != cudaSuccess) s = KO_ERR_CUDA;
    }
    if (!s) s = ko_model_check(md);
    if (!s) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (gpu_ms) *gpu_ms = ms;
        long long bi = 0;
        s = best_of(top_ms, top_k, best_makespan, &bi);
        int8_t r[kMaxK];
        if (!s && cudaMemcpy(r, top_rows + (size_t)bi * kMaxK, kMaxK, cudaMemcpyDeviceToHost) != cudaSuccess)
            s = KO_ERR_CUDA;
        if (!s)
            for (int i = 0; i < h.n; i++) best_order[i] = r[i];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(rows); cudaFree(top_rows); cudaFree(y_all); cudaFree(top_idx); cudaFree(top_ms);
    cudaFree(sel_state); cudaFree(sel_hist); cudaFree(sel_cnt); cudaFree(d_chunk);
    return s;
}

// Surrogate-guided local search.  Screening: the network scores n_cand
// uniform random orders, the top_k are rescored exactly, and the `beam` best
// exact orders seed the search.  Each round: every swap and every single move
// of each beam order is scored by the network, the k2 best are rescored
// exactly, and the beam becomes the `beam` best distinct orders seen so far.
// Every reported makespan is exact.
ko_status ko_model_search_set(ko_model *md, const KoSet &h, long long n_cand, int top_k, int rounds, int beam,
                              uint64_t seed, int32_t *best_order, int64_t *best_makespan, double *gpu_ms,
                              cudaStream_t st)
{
    const int n = h.n;
    if (n_cand < 1 || top_k < 1 || top_k > n_cand || n_cand > (1ll << 26) || rounds < 0 || rounds > 1024 ||
        beam < 1 || beam > 64 || n < 2)
        return KO_ERR_ARG;
    if (!ko_fast_applicable(h)) return KO_ERR_OVERFLOW;
    const KoSet *hs[1] = {&h};
    SetTables tb;
    ko_status s = build_tables(hs, 1, &tb, st);
    if (s) return s;
    const int C = md->chunk;
    const int k2 = 256;
    const long long padded = (n_cand + C - 1) / C * C;
    const int per = n * (n - 1) / 2 + n * (n - 1);
    const int nb_rows = beam * per, nb_pad = (nb_rows + 127) / 128 * 128;
    const int kmax = top_k > k2 ? top_k : k2;
    int8_t *rows = nullptr, *top_rows = nullptr, *nb = nullptr, *base = nullptr;
    float *y_all = nullptr;
    int *top_idx = nullptr;
    int64_t *top_ms = nullptr;
    uint32_t *sel_state = nullptr;
    unsigned int *sel_hist = nullptr, *sel_cnt = nullptr;
    KoChunk *d_chunk = nullptr;
    if (!dalloc(&rows, (size_t)padded * kMaxK) || !dalloc(&y_all, (size_t)std::max<long long>(n_cand, nb_pad)) ||
        !dalloc(&top_idx, kmax) || !dalloc(&top_rows, (size_t)kmax * kMaxK) || !dalloc(&top_ms, kmax) ||
        !dalloc(&nb, (size_t)nb_pad * kMaxK) || !dalloc(&base, (size_t)beam * kMaxK) || !dalloc(&sel_state, 2) ||
        !dalloc(&sel_hist, 256) || !dalloc(&sel_cnt, 2) || !dalloc(&d_chunk, 1))
        s = KO_ERR_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    struct Cand {
        int64_t ms;
        std::vector<int8_t> row;
    };
    std::vector<Cand> pool;
    // exact makespans of `cnt` device rows -> pool
    auto collect = [&](int cnt) -> ko_status {
        std::vector<int64_t> hm(cnt);
        std::vector<int8_t> hr((size_t)cnt * kMaxK);
        if (cudaMemcpyAsync(hm.data(), top_ms, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hr.data(), top_rows, hr.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return KO_ERR_CUDA;
        for (int i = 0; i < cnt; i++)
            if (hm[i] >= 0) pool.push_back(Cand{hm[i], std::vector<int8_t>(hr.begin() + (size_t)i * kMaxK, hr.begin() + (size_t)(i + 1) * kMaxK)});
        std::stable_sort(pool.begin(), pool.end(), [](const Cand &a, const Cand &b) { return a.ms < b.ms; });
        std::vector<Cand> kept;
        for (const Cand &c : pool) {
            bool dup = false;
            for (const Cand &k : kept) dup = dup || k.row == c.row;
            if (!dup) kept.push_back(c);
            if ((int)kept.size() == beam) break;
        }
        pool.swap(kept);
        return KO_OK;
    };
    if (!s) s = make_events(&e0, &e1);
    if (!s) s = ensure_acts(md, C);
    if (!s) {
        cudaEventRecord(e0, st);
        // screening
        if (cudaMemsetAsync(rows, 0, (size_t)padded * kMaxK, st) != cudaSuccess ||
            cudaMemsetAsync(nb, 0, (size_t)nb_pad * kMaxK, st) != cudaSuccess)
            s = KO_ERR_CUDA;
        if (!s) s = cuda_ok(ko_mlp_random_orders(rows, kMaxK, n_cand, n, mix64(seed ^ 0xC0FFEEull), st));
        for (long long off = 0; off < n_cand && !s; off += C) {
            const long long c = n_cand - off < C ? n_cand - off : C;
            if ((s = cuda_ok(ko_mlp_encode(rows + (size_t)off * kMaxK, kMaxK, nullptr, nullptr, tb.set_n, tb.kfeat,
                                           tb.gfeat, C, md->a0, nullptr, st))))
                break;
            if ((s = forward(md, C, false, st))) break;
            if (cudaMemcpyAsync(y_all + off, md->y, sizeof(float) * c, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                s = KO_ERR_CUDA;
        }
        if (!s) s = cuda_ok(ko_mlp_topk(y_all, n_cand, top_k, sel_state, sel_hist, sel_cnt, top_idx, st));
        if (!s) s = cuda_ok(ko_mlp_gather_rows(rows, kMaxK, top_idx, top_k, top_rows, st));
        if (!s) s = exact_rows(&md->fast, tb.sets, h, 0, top_rows, top_k, top_ms, d_chunk, st);
        if (!s) s = collect(top_k);
        // local search rounds
        for (int r = 0; r < rounds && !s && !pool.empty(); r++) {
            const int nbase = (int)pool.size();
            std::vector<int8_t> hb((size_t)nbase * kMaxK);
            for (int i = 0; i < nbase; i++) std::memcpy(&hb[(size_t)i * kMaxK], pool[i].row.data(), kMaxK);
            if (cudaMemcpyAsync(base, hb.data(), hb.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) { s = KO_ERR_CUDA; break; }
            if ((s = cuda_ok(ko_mlp_neighbours(base, nbase, n, nb, st)))) break;
            const int q = nbase * per, qpad = (q + 127) / 128 * 128;
            for (int off = 0; off < qpad && !s; off += C) {
                const int c = qpad - off < C ? qpad - off : C;
                if ((s = cuda_ok(ko_mlp_encode(nb + (size_t)off * kMaxK, kMaxK, nullptr, nullptr, tb.set_n, tb.kfeat,
                                               tb.gfeat, c, md->a0, nullptr, st))))
                    break;
                if ((s = forward(md, c, false, st))) break;
                if (cudaMemcpyAsync(y_all + off, md->y, sizeof(float) * c, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    s = KO_ERR_CUDA;
            }
            const int kk = q < k2 ? q : k2;
            if (!s) s = cuda_ok(ko_mlp_topk(y_all, q, kk, sel_state, sel_hist, sel_cnt, top_idx, st));
            if (!s) s = cuda_ok(ko_mlp_gather_rows(nb, kMaxK, top_idx, kk, top_rows, st));
            if (!s) s = exact_rows(&md->fast, tb.sets, h, 0, top_rows, kk, top_ms, d_chunk, st);
            if (!s) s = collect(kk);
        }
        // exact steepest descent from the best exact order (the simulator alone decides)
        if (!s && md->polish > 0 && !pool.empty()) {
            if (cudaStreamSynchronize(st) != cudaSuccess) s = KO_ERR_CUDA;
            std::vector<int32_t> start(n), out(n);
            for (int i = 0; i < n; i++) start[i] = pool[0].row[i];
            int64_t pms = -1, evals = 0;
            int32_t steps = 0;
            double lms = 0.0;
            if (!s) s = ko_local_search_set(&md->fast, h, start.data(), true, md->polish, out.data(), &pms, &steps,
                                            &evals, &lms, st);
            if (!s && pms >= 0 && pms < pool[0].ms) {
                pool[0].ms = pms;
                for (int i = 0; i < n; i++) pool[0].row[i] = (int8_t)out[i];
            }
        }
        cudaEventRecord(e1, st);
        if (!s && cudaStreamSynchronize(st) != cudaSuccess) s = KO_ERR_CUDA;
    }
    if (!s) s = ko_model_check(md);
    if (!s && pool.empty()) s = KO_ERR_STATE;
    if (!s) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (gpu_ms) *gpu_ms = ms;
        *best_makespan = pool[0].ms;
        for (int i = 0; i < n; i++) best_order[i] = pool[0].row[i];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(rows); cudaFree(top_rows); cudaFree(nb); cudaFree(base); cudaFree(y_all); cudaFree(top_idx);
    cudaFree(top_ms); cudaFree(sel_state); cudaFree(sel_hist); cudaFree(sel_cnt); cudaFree(d_chunk);
    return s;
}

ko_status ko_random_search_set(KoFastState *fs, const KoSet &h, long long n_orders, uint64_t seed,
                               int32_t *best_order, int64_t *best_makespan, double *gpu_ms, cudaStream_t st)
{
    if (n_orders < 1 || n_orders > (1ll << 26)) return KO_ERR_ARG;
    if (!ko_fast_applicable(h)) return KO_ERR_OVERFLOW;
    const KoSet *hs[1] = {&h};
    SetTables tb;
    ko_status s = build_tables(hs, 1, &tb, st);
    if (s) return s;
    int8_t *rows = nullptr;
    int64_t *ms = nullptr;
    KoChunk *d_chunk = nullptr;
    if (!dalloc(&rows, (size_t)n_orders * kMaxK) || !dalloc(&ms, (size_t)n_orders) || !dalloc(&d_chunk, 1))
        s = KO_ERR_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!s) s = make_events(&e0, &e1);
    if (!s) {
        cudaEventRecord(e0, st);
        s = cuda_ok(ko_mlp_random_orders(rows, kMaxK, n_orders, h.n, mix64(seed ^ 0xBEEFull), st));
        if (!s) s = exact_rows(fs, tb.sets, h, 0, rows, n_orders, ms, d_chunk, st);
        cudaEventRecord(e1, st);
        if (!s && cudaStreamSynchronize(st) != cudaSuccess) s = KO_ERR_CUDA;
    }
    if (!s) {
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (gpu_ms) *gpu_ms = t;
        long long bi = 0;
        s = best_of(ms, n_orders, best_makespan, &bi);
        int8_t r[kMaxK];
        if (!s && cudaMemcpy(r, rows + (size_t)bi * kMaxK, kMaxK, cudaMemcpyDeviceToHost) != cudaSuccess)
            s = KO_ERR_CUDA;
        if (!s)
            for (int i = 0; i < h.n; i++) best_order[i] = r[i];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(rows); cudaFree(ms); cudaFree(d_chunk);
    return s;
}

// Steepest-descent hill climbing with exact scoring.  Neighbours of the
// current order come from the neighbours kernel (swaps of two positions, then
// moves of one kernel to another position); every one is simulated exactly,
// the lowest makespan wins (lowest neighbour index among equals) and the walk
// moves only on a strict improvement.  One step = one H2D of the current order,
// two launches and one D2H of the neighbours' makespans.
ko_status ko_local_search_set(KoFastState *fs, const KoSet &h, const int32_t *start, bool moves, int max_iters,
                              int32_t *order_out, int64_t *makespan_out, int32_t *steps_out, int64_t *evals_out,
                              double *gpu_ms, cudaStream_t st)
{
    const int n = h.n;
    if (n < 1 || max_iters < 0 || max_iters > (1 << 20)) return KO_ERR_ARG;
    if (!ko_fast_applicable(h)) return KO_ERR_OVERFLOW;
    std::vector<int8_t> cur(kMaxK, 0);
    {
        std::vector<char> seen(n, 0);
        for (int i = 0; i < n; i++) {
            if (start[i] < 0 || start[i] >= n || seen[start[i]]) return KO_ERR_ARG;
            seen[start[i]] = 1;
            cur[i] = (int8_t)start[i];
        }
    }
    const KoSet *hs[1] = {&h};
    SetTables tb;
    ko_status s = build_tables(hs, 1, &tb, st);
    if (s) return s;
    const int swaps = n * (n - 1) / 2, per = swaps + n * (n - 1);
    const int nq = moves ? per : swaps;
    int8_t *base = nullptr, *nb = nullptr;
    int64_t *ms = nullptr;
    KoChunk *d_chunk = nullptr;
    if (!dalloc(&base, kMaxK) || !dalloc(&nb, (size_t)(per > 0 ? per : 1) * kMaxK) ||
        !dalloc(&ms, (size_t)(per > 0 ? per : 1) + 1) || !dalloc(&d_chunk, 1))
        s = KO_ERR_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int64_t cur_ms = -1, evals = 0;
    int steps = 0;
    std::vector<int64_t> hm((size_t)(nq > 0 ? nq : 1));
    if (!s) s = make_events(&e0, &e1);
    if (!s) {
        cudaEventRecord(e0, st);
        if (cudaMemcpyAsync(base, cur.data(), kMaxK, cudaMemcpyHostToDevice, st) != cudaSuccess) s = KO_ERR_CUDA;
        if (!s) s = exact_rows(fs, tb.sets, h, 0, base, 1, ms + per, d_chunk, st);
        if (!s && (cudaMemcpyAsync(&cur_ms, ms + per, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                   cudaStreamSynchronize(st) != cudaSuccess))
            s = KO_ERR_CUDA;
        if (!s && cur_ms < 0) s = KO_ERR_STATE;
        evals = 1;
        while (!s && steps < max_iters && nq > 0) {
            if (cudaMemcpyAsync(base, cur.data(), kMaxK, cudaMemcpyHostToDevice, st) != cudaSuccess) { s = KO_ERR_CUDA; break; }
            if ((s = cuda_ok(ko_mlp_neighbours(base, 1, n, nb, st)))) break;
            if ((s = exact_rows(fs, tb.sets, h, 0, nb, nq, ms, d_chunk, st))) break;
            if (cudaMemcpyAsync(hm.data(), ms, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { s = KO_ERR_CUDA; break; }
            evals += nq;
            int bq = -1;
            for (int q = 0; q < nq; q++) {
                if (hm[q] < 0) { s = KO_ERR_STATE; break; }
                if (bq < 0 || hm[q] < hm[bq]) bq = q;
            }
            if (s || hm[bq] >= cur_ms) break;
            if (cudaMemcpy(cur.data(), nb + (size_t)bq * kMaxK, kMaxK, cudaMemcpyDeviceToHost) != cudaSuccess) { s = KO_ERR_CUDA; break; }
            cur_ms = hm[bq];
            steps++;
        }
        cudaEventRecord(e1, st);
        if (!s && cudaStreamSynchronize(st) != cudaSuccess) s = KO_ERR_CUDA;
    }
    if (!s) {
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (gpu_ms) *gpu_ms = t;
        for (int i = 0; i < n; i++) order_out[i] = cur[i];
        *makespan_out = cur_ms;
        if (steps_out) *steps_out = steps;
        if (evals_out) *evals_out = evals;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(base); cudaFree(nb); cudaFree(ms); cudaFree(d_chunk);
    return s;
}

// Features of explicit orders of one set (encoder output as floats), for tests.
ko_status ko_model_features(const KoSet &h, const int8_t *orders, long long n, float *x_out, cudaStream_t st)
{
    const KoSet *hs[1] = {&h};
    SetTables tb;
    ko_status s = build_tables(hs, 1, &tb, st);
    if (s) return s;
    int8_t *rows = nullptr;
    uint16_t *x = nullptr;
    if (!dalloc(&rows, (size_t)n * kMaxK) || !dalloc(&x, (size_t)n * kMlpIn)) {
        cudaFree(rows);
        return KO_ERR_NOMEM;
    }
    std::vector<int8_t> hr((size_t)n * kMaxK, 0);
    for (long long i = 0; i < n; i++) std::memcpy(&hr[(size_t)i * kMaxK], orders + (size_t)i * h.n, h.n);
    std::vector<uint16_t> hx((size_t)n * kMlpIn);
    if (cudaMemcpyAsync(rows, hr.data(), hr.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) s = KO_ERR_CUDA;
    if (!s) s = cuda_ok(ko_mlp_encode(rows, kMaxK, nullptr, nullptr, tb.set_n, tb.kfeat, tb.gfeat, (int)n, x, nullptr, st));
    if (!s && (cudaMemcpyAsync(hx.data(), x, hx.size() * 2, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess))
        s = KO_ERR_CUDA;
    if (!s)
        for (size_t i = 0; i < hx.size(); i++) {
            const uint32_t u = (uint32_t)hx[i] << 16;
            std::memcpy(&x_out[i], &u, 4);
        }
    cudaFree(rows);
    cudaFree(x);
    return s;
}
