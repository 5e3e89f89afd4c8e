// Learned selector: a fully connected 16 -> H1 -> H2 -> K network with ReLU
// that maps the Table 1 feature vector (Section 3.2.2) to a variant.  The
// paper builds its feature-based classifier with a decision tree or naive
// Bayes; this library trains a small MLP on the GPU with the kernels below
// (forward, softmax cross-entropy backward, Adam), and keeps the paper's
// profiling rule (Section 3.2.1) as its fallback when the network's top two
// logits are close.
//
// Parameters are packed row-major as W1[H1][16], b1[H1], W2[H2][H1], b2[H2],
// W3[K][H2], b3[K] (float).  Inputs are standardised as
// z = (v - mean) * istd, each operation rounded to float.  Every dot product
// is a chain of fmaf starting from the bias, inputs in ascending order: the
// same order on the host and the device, so logits agree bit for bit.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"

struct spmv_model {
    int32_t h1 = 0, h2 = 0, k = 0;
    float mean[16] = {}, istd[16] = {};
    std::vector<float> params;
    std::vector<int32_t> variants;
    float min_margin = 0.f;
    // optional launch parameters per output: threads_per_row, block_nnz,
    // items_per_warp (a second-level model choosing among one variant's
    // launch configurations); empty when the model names variants only
    std::vector<int32_t> launch;
};

namespace spmvlib {
namespace {

constexpr int kMaxH = 256;       // hidden width limit of the forward kernels
constexpr int kTrainMaxH = 128;  // hidden width limit of training
constexpr int kMaxK = 32;

__host__ __device__ __forceinline__ int64_t n_params(int h1, int h2, int k)
{
    return (int64_t)h1 * 16 + h1 + (int64_t)h2 * h1 + h2 + (int64_t)k * h2 + k;
}

// ---- host forward (spmv_select_model) ---------------------------------------
void host_forward(const spmv_model& m, const float* v, float* logits)
{
    const float* W1 = m.params.data();
    const float* b1 = W1 + m.h1 * 16;
    const float* W2 = b1 + m.h1;
    const float* b2 = W2 + m.h2 * m.h1;
    const float* W3 = b2 + m.h2;
    const float* b3 = W3 + m.k * m.h2;
    float z[16], a1[kMaxH], a2[kMaxH];
    for (int i = 0; i < 16; ++i) {
        volatile float d = v[i] - m.mean[i];  // keep the two roundings separate
        z[i] = d * m.istd[i];
    }
    for (int o = 0; o < m.h1; ++o) {
        float acc = b1[o];
        for (int i = 0; i < 16; ++i) acc = fmaf(W1[o * 16 + i], z[i], acc);
        a1[o] = acc > 0.f ? acc : 0.f;
    }
    for (int o = 0; o < m.h2; ++o) {
        float acc = b2[o];
        for (int i = 0; i < m.h1; ++i) acc = fmaf(W2[o * m.h1 + i], a1[i], acc);
        a2[o] = acc > 0.f ? acc : 0.f;
    }
    for (int o = 0; o < m.k; ++o) {
        float acc = b3[o];
        for (int i = 0; i < m.h2; ++i) acc = fmaf(W3[o * m.h2 + i], a2[i], acc);
        logits[o] = acc;
    }
}

// ---- device kernels -----------------------------------------------------------
struct Net {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
    int h1, h2, k;
};
__device__ __forceinline__ Net unpack(const float* p, int h1, int h2, int k)
{
    Net n;
    n.W1 = p; n.b1 = n.W1 + h1 * 16; n.W2 = n.b1 + h1; n.b2 = n.W2 + h2 * h1;
    n.W3 = n.b2 + h2; n.b3 = n.W3 + k * h2;
    n.h1 = h1; n.h2 = h2; n.k = k;
    return n;
}

// One sample per thread; weights read through the read-only path.
__global__ void k_mlp_forward(const float* __restrict__ params, const float* __restrict__ mean,
                              const float* __restrict__ istd, int h1, int h2, int k,
                              const float* __restrict__ v, int n, float* __restrict__ logits)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const Net N = unpack(params, h1, h2, k);
    float z[16], a1[kMaxH], a2[kMaxH];
    for (int i = 0; i < 16; ++i) z[i] = __fmul_rn(__fsub_rn(v[s * 16 + i], mean[i]), istd[i]);
    for (int o = 0; o < h1; ++o) {
        float acc = __ldg(N.b1 + o);
        for (int i = 0; i < 16; ++i) acc = __fmaf_rn(__ldg(N.W1 + o * 16 + i), z[i], acc);
        a1[o] = acc > 0.f ? acc : 0.f;
    }
    for (int o = 0; o < h2; ++o) {
        float acc = __ldg(N.b2 + o);
        for (int i = 0; i < h1; ++i) acc = __fmaf_rn(__ldg(N.W2 + o * h1 + i), a1[i], acc);
        a2[o] = acc > 0.f ? acc : 0.f;
    }
    for (int o = 0; o < k; ++o) {
        float acc = __ldg(N.b3 + o);
        for (int i = 0; i < h2; ++i) acc = __fmaf_rn(__ldg(N.W3 + o * h2 + i), a2[i], acc);
        logits[s * k + o] = acc;
    }
}

// Mean softmax cross-entropy over the batch and its gradient.  Each CTA
// takes a contiguous slice of at most kSlice samples: it runs their forward
// and backward passes in shared memory, then every thread accumulates the
// gradient entries it owns over the slice's samples in order and writes the
// CTA's partial gradient; k_mlp_reduce sums the partials in CTA order.  The
// result is deterministic.
constexpr int kSlice = 32;
constexpr int kMT = 256;

struct __align__(16) TrainSmem {
    float z[kSlice][16];
    float a1[kSlice][kTrainMaxH];
    float a2[kSlice][kTrainMaxH];
    float d1[kSlice][kTrainMaxH];
    float d2[kSlice][kTrainMaxH];
    float d3[kSlice][kMaxK];
    float loss[kSlice];
};

__global__ void __launch_bounds__(kMT)
k_mlp_loss_grad(const float* __restrict__ params, int h1, int h2, int k,
                const float* __restrict__ z, const int32_t* __restrict__ labels,
                const float* __restrict__ q, int n, float* __restrict__ part,
                float* __restrict__ part_loss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& sm = *reinterpret_cast<TrainSmem*>(smem_raw);
    const Net N = unpack(params, h1, h2, k);
    const int s0 = blockIdx.x * kSlice;
    const int ns = min(kSlice, n - s0);
    const int tid = threadIdx.x;
    for (int t = tid; t < ns * 16; t += kMT) sm.z[t / 16][t % 16] = z[(s0 + t / 16) * 16 + t % 16];
    __syncthreads();
    for (int t = tid; t < ns * h1; t += kMT) {
        const int s = t / h1, o = t % h1;
        float acc = N.b1[o];
        for (int i = 0; i < 16; ++i) acc = __fmaf_rn(N.W1[o * 16 + i], sm.z[s][i], acc);
        sm.a1[s][o] = acc > 0.f ? acc : 0.f;
    }
    __syncthreads();
    for (int t = tid; t < ns * h2; t += kMT) {
        const int s = t / h2, o = t % h2;
        float acc = N.b2[o];
        for (int i = 0; i < h1; ++i) acc = __fmaf_rn(N.W2[o * h1 + i], sm.a1[s][i], acc);
        sm.a2[s][o] = acc > 0.f ? acc : 0.f;
    }
    __syncthreads();
    for (int t = tid; t < ns * k; t += kMT) {
        const int s = t / k, o = t % k;
        float acc = N.b3[o];
        for (int i = 0; i < h2; ++i) acc = __fmaf_rn(N.W3[o * h2 + i], sm.a2[s][i], acc);
        sm.d3[s][o] = acc;  // logits for now
    }
    __syncthreads();
    // softmax cross-entropy per sample; d3 = (p - onehot) / n, or with a
    // target distribution q: loss = -sum q_o log p_o, d3 = (p S - q) / n
    // where S = sum q_o
    if (tid < ns) {
        const int s = tid;
        float mx = -INFINITY;
        for (int o = 0; o < k; ++o) mx = fmaxf(mx, sm.d3[s][o]);
        float den = 0.f;
        for (int o = 0; o < k; ++o) den += expf(sm.d3[s][o] - mx);
        if (q == nullptr) {
            const int y = labels[s0 + s];
            sm.loss[s] = -(sm.d3[s][y] - mx - logf(den));
            for (int o = 0; o < k; ++o) {
                const float p = expf(sm.d3[s][o] - mx) / den;
                sm.d3[s][o] = (p - (o == y ? 1.f : 0.f)) / (float)n;
            }
        } else {
            const float* qs = q + (int64_t)(s0 + s) * k;
            const float lse = mx + logf(den);
            float S = 0.f, l = 0.f;
            for (int o = 0; o < k; ++o) {
                S += qs[o];
                l -= qs[o] * (sm.d3[s][o] - lse);
            }
            sm.loss[s] = l;
            for (int o = 0; o < k; ++o) {
                const float p = expf(sm.d3[s][o] - lse);
                sm.d3[s][o] = (p * S - qs[o]) / (float)n;
            }
        }
    }
    __syncthreads();
    for (int t = tid; t < ns * h2; t += kMT) {
        const int s = t / h2, i = t % h2;
        float acc = 0.f;
        for (int o = 0; o < k; ++o) acc = __fmaf_rn(N.W3[o * h2 + i], sm.d3[s][o], acc);
        sm.d2[s][i] = sm.a2[s][i] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    for (int t = tid; t < ns * h1; t += kMT) {
        const int s = t / h1, i = t % h1;
        float acc = 0.f;
        for (int o = 0; o < h2; ++o) acc = __fmaf_rn(N.W2[o * h1 + i], sm.d2[s][o], acc);
        sm.d1[s][i] = sm.a1[s][i] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // per-CTA gradient partials, each entry owned by one thread
    const int64_t P = n_params(h1, h2, k);
    float* g = part + (int64_t)blockIdx.x * P;
    float* gW1 = g;
    float* gb1 = gW1 + h1 * 16;
    float* gW2 = gb1 + h1;
    float* gb2 = gW2 + h2 * h1;
    float* gW3 = gb2 + h2;
    float* gb3 = gW3 + k * h2;
    for (int e = tid; e < h1 * 16; e += kMT) {
        const int o = e / 16, i = e % 16;
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc = __fmaf_rn(sm.d1[s][o], sm.z[s][i], acc);
        gW1[e] = acc;
    }
    for (int e = tid; e < h1; e += kMT) {
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += sm.d1[s][e];
        gb1[e] = acc;
    }
    for (int e = tid; e < h2 * h1; e += kMT) {
        const int o = e / h1, i = e % h1;
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc = __fmaf_rn(sm.d2[s][o], sm.a1[s][i], acc);
        gW2[e] = acc;
    }
    for (int e = tid; e < h2; e += kMT) {
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += sm.d2[s][e];
        gb2[e] = acc;
    }
    for (int e = tid; e < k * h2; e += kMT) {
        const int o = e / h2, i = e % h2;
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc = __fmaf_rn(sm.d3[s][o], sm.a2[s][i], acc);
        gW3[e] = acc;
    }
    for (int e = tid; e < k; e += kMT) {
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += sm.d3[s][e];
        gb3[e] = acc;
    }
    if (tid == 0) {
        float l = 0.f;
        for (int s = 0; s < ns; ++s) l += sm.loss[s];
        part_loss[blockIdx.x] = l;
    }
}

__global__ void k_mlp_reduce(const float* __restrict__ part, const float* __restrict__ part_loss,
                             int n_parts, int64_t P, int n, float* __restrict__ grad,
                             float* __restrict__ loss)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < P) {
        float acc = 0.f;
        for (int c = 0; c < n_parts; ++c) acc += part[(int64_t)c * P + e];
        grad[e] = acc;
    }
    if (e == 0) {
        float l = 0.f;
        for (int c = 0; c < n_parts; ++c) l += part_loss[c];
        *loss = l / (float)n;
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float wd, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // each operation rounded separately (no contraction), as the definition reads
    const float gi = g[i];
    const float mi = __fadd_rn(__fmul_rn(b1, m[i]), __fmul_rn(__fsub_rn(1.f, b1), gi));
    const float vi = __fadd_rn(__fmul_rn(b2, v[i]), __fmul_rn(__fsub_rn(1.f, b2), __fmul_rn(gi, gi)));
    m[i] = mi;
    v[i] = vi;
    const float mh = __fdiv_rn(mi, c1), vh = __fdiv_rn(vi, c2);
    const float step = __fadd_rn(__fdiv_rn(mh, __fadd_rn(__fsqrt_rn(vh), eps)), __fmul_rn(wd, p[i]));
    p[i] = __fsub_rn(p[i], __fmul_rn(lr, step));
}

}  // namespace
}  // namespace spmvlib

using namespace spmvlib;

namespace {

bool shape_ok(int h1, int h2, int k, int max_h)
{
    return h1 >= 1 && h2 >= 1 && h1 <= max_h && h2 <= max_h && k >= 2 && k <= kMaxK;
}

const char kMagic[8] = {'S', 'P', 'M', 'V', 'M', 'L', 'P', '1'};
const char kMagic2[8] = {'S', 'P', 'M', 'V', 'M', 'L', 'P', '2'};  // + launch parameters

// output o's launch parameters as a choice of its variant (validated)
spmv_status launch_choice(const spmv_model_t* m, int o, spmv_choice_t* c)
{
    c->variant = m->variants[o];
    c->threads_per_row = m->launch[3 * o];
    c->block_nnz = m->launch[3 * o + 1];
    c->items_per_warp = m->launch[3 * o + 2];
    c->value_type = SPMV_VAL_F64;
    return check_choice(c);
}

}  // namespace

extern "C" {

spmv_status spmv_model_create(int32_t h1, int32_t h2, int32_t k, const float* mean,
                              const float* istd, const float* params, const int32_t* variants,
                              float min_margin, spmv_model_t** out)
{
    clear_error();
    if (!out || !mean || !istd || !params || !variants)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_model_create: NULL argument");
    *out = nullptr;
    if (!shape_ok(h1, h2, k, kMaxH)) return fail(SPMV_ERR_MODEL, "model shape out of range");
    for (int o = 0; o < k; ++o)
        if (variants[o] < 0 || variants[o] >= SPMV_NUM_VARIANTS)
            return fail(SPMV_ERR_MODEL, "model names an unknown variant");
    spmv_model* m = new (std::nothrow) spmv_model();
    if (!m) return fail(SPMV_ERR_NOMEM, "host allocation failed");
    m->h1 = h1; m->h2 = h2; m->k = k;
    memcpy(m->mean, mean, sizeof(m->mean));
    memcpy(m->istd, istd, sizeof(m->istd));
    m->params.assign(params, params + n_params(h1, h2, k));
    m->variants.assign(variants, variants + k);
    m->min_margin = min_margin;
    for (float p : m->params)
        if (!isfinite(p)) { delete m; return fail(SPMV_ERR_MODEL, "non-finite model parameter"); }
    *out = m;
    return SPMV_OK;
}

spmv_status spmv_model_set_launch(spmv_model_t* m, const int32_t* launch)
{
    clear_error();
    if (!m || !launch) return fail(SPMV_ERR_INVALID_ARG, "spmv_model_set_launch: NULL argument");
    std::vector<int32_t> keep;
    keep.swap(m->launch);
    m->launch.assign(launch, launch + 3 * m->k);
    for (int o = 0; o < m->k; ++o) {
        spmv_choice_t c = {};
        if (launch_choice(m, o, &c) != SPMV_OK) {
            m->launch.swap(keep);
            return fail(SPMV_ERR_MODEL, "launch parameters not valid for the output's variant");
        }
    }
    return SPMV_OK;
}

spmv_status spmv_model_save(const spmv_model_t* m, const char* path)
{
    clear_error();
    if (!m || !path) return fail(SPMV_ERR_INVALID_ARG, "spmv_model_save: NULL argument");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(SPMV_ERR_INVALID_ARG, std::string("cannot open ") + path);
    const int32_t hdr[3] = {m->h1, m->h2, m->k};
    const bool v2 = !m->launch.empty();
    bool ok = fwrite(v2 ? kMagic2 : kMagic, 1, 8, f) == 8 && fwrite(hdr, 4, 3, f) == 3 &&
              fwrite(m->mean, 4, 16, f) == 16 && fwrite(m->istd, 4, 16, f) == 16 &&
              fwrite(m->params.data(), 4, m->params.size(), f) == m->params.size() &&
              fwrite(m->variants.data(), 4, m->variants.size(), f) == m->variants.size() &&
              fwrite(&m->min_margin, 4, 1, f) == 1;
    if (v2) ok = ok && fwrite(m->launch.data(), 4, m->launch.size(), f) == m->launch.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? SPMV_OK : fail(SPMV_ERR_INVALID_ARG, std::string("write failed: ") + path);
}

spmv_status spmv_model_load(const char* path, spmv_model_t** out)
{
    clear_error();
    if (!path || !out) return fail(SPMV_ERR_INVALID_ARG, "spmv_model_load: NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(SPMV_ERR_MODEL, std::string("cannot open model file ") + path);
    char magic[8];
    int32_t hdr[3];
    float mean[16], istd[16], margin = 0.f;
    std::vector<float> params;
    std::vector<int32_t> variants, launch;
    bool ok = fread(magic, 1, 8, f) == 8 && (memcmp(magic, kMagic, 8) == 0 || memcmp(magic, kMagic2, 8) == 0) &&
              fread(hdr, 4, 3, f) == 3 && shape_ok(hdr[0], hdr[1], hdr[2], kMaxH);
    const bool v2 = ok && memcmp(magic, kMagic2, 8) == 0;
    if (ok) {
        params.resize((size_t)n_params(hdr[0], hdr[1], hdr[2]));
        variants.resize((size_t)hdr[2]);
        ok = fread(mean, 4, 16, f) == 16 && fread(istd, 4, 16, f) == 16 &&
             fread(params.data(), 4, params.size(), f) == params.size() &&
             fread(variants.data(), 4, variants.size(), f) == variants.size() &&
             fread(&margin, 4, 1, f) == 1;
        if (ok && v2) {
            launch.resize(3 * (size_t)hdr[2]);
            ok = fread(launch.data(), 4, launch.size(), f) == launch.size();
        }
        char extra;
        if (ok && fread(&extra, 1, 1, f) != 0) ok = false;  // trailing bytes: corrupt
    }
    fclose(f);
    if (!ok) return fail(SPMV_ERR_MODEL, std::string("corrupt or truncated model file ") + path);
    spmv_status st = spmv_model_create(hdr[0], hdr[1], hdr[2], mean, istd, params.data(), variants.data(),
                                       margin, out);
    if (st != SPMV_OK || !v2) return st;
    if ((st = spmv_model_set_launch(*out, launch.data())) != SPMV_OK) {
        spmv_model_free(*out);
        *out = nullptr;
    }
    return st;
}

void spmv_model_free(spmv_model_t* m) { delete m; }

spmv_status spmv_model_logits(const spmv_model_t* m, const float* vec16, float* logits)
{
    clear_error();
    if (!m || !vec16 || !logits) return fail(SPMV_ERR_INVALID_ARG, "spmv_model_logits: NULL argument");
    host_forward(*m, vec16, logits);
    return SPMV_OK;
}

spmv_status spmv_select_model(const spmv_features_t* f, const spmv_model_t* m,
                              const spmv_profile_t* p, const spmv_thresholds_t* th,
                              spmv_choice_t* out)
{
    clear_error();
    if (!f || !m || !out) return fail(SPMV_ERR_INVALID_ARG, "spmv_select_model: NULL argument");
    float logits[kMaxK];
    host_forward(*m, f->vec, logits);
    int best = 0;
    for (int o = 1; o < m->k; ++o)
        if (logits[o] > logits[best]) best = o;
    float second = -INFINITY;
    for (int o = 0; o < m->k; ++o)
        if (o != best && logits[o] > second) second = logits[o];
    spmv_choice_t c = {};
    c.variant = m->variants[best];
    if (!m->launch.empty()) {
        spmv_status st = launch_choice(m, best, &c);
        if (st != SPMV_OK) return st;
    }
    c.cls = -1;
    c.value_type = SPMV_VAL_F64;
    c.margin = logits[best] - second;
    c.source = 2;
    if (c.margin < m->min_margin && p) {
        int32_t cls = -1;
        spmv_status st = spmv_classify_profile(p, th, &cls);
        if (st != SPMV_OK) return st;
        const float margin = c.margin;
        if ((st = spmv_class_choice(cls, &c)) != SPMV_OK) return st;
        c.margin = margin;
        c.used_fallback = 1;
    }
    *out = c;
    return SPMV_OK;
}

spmv_status spmv_select_model_refined(const spmv_features_t* f, const spmv_model_t* m,
                                      const spmv_model_t* sub, const spmv_profile_t* p,
                                      const spmv_thresholds_t* th, spmv_choice_t* out)
{
    spmv_status st = spmv_select_model(f, m, p, th, out);
    if (st != SPMV_OK || !sub || sub->launch.empty() || out->used_fallback) return st;
    for (int o = 0; o < sub->k; ++o)
        if (sub->variants[o] != out->variant) return SPMV_OK;  // another variant: first level only
    spmv_choice_t c2;
    if ((st = spmv_select_model(f, sub, nullptr, nullptr, &c2)) != SPMV_OK) return st;
    out->threads_per_row = c2.threads_per_row;
    out->block_nnz = c2.block_nnz;
    out->items_per_warp = c2.items_per_warp;
    return SPMV_OK;
}

spmv_status spmv_mlp_forward(const float* params, const float* mean, const float* istd,
                             int32_t h1, int32_t h2, int32_t k, const float* v, int32_t n,
                             float* logits, spmv_stream_t stream)
{
    clear_error();
    if (!shape_ok(h1, h2, k, kMaxH) || n < 0) return fail(SPMV_ERR_INVALID_ARG, "bad MLP shape");
    if (n == 0) return SPMV_OK;
    if (!params || !mean || !istd || !v || !logits)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_mlp_forward: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_mlp_forward<<<(n + 63) / 64, 64, 0, s>>>(params, mean, istd, h1, h2, k, v, n, logits);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

namespace {
spmv_status loss_grad_impl(const float* params, int32_t h1, int32_t h2, int32_t k,
                           const float* z, const int32_t* labels, const float* q, int32_t n,
                           float* grad, float* loss, spmv_stream_t stream)
{
    clear_error();
    if (!shape_ok(h1, h2, k, kTrainMaxH) || n <= 0)
        return fail(SPMV_ERR_INVALID_ARG, "bad MLP training shape (hidden <= 128, k <= 32)");
    if (!params || !z || (!labels && !q) || !grad || !loss)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_mlp_loss_grad: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int parts = (n + kSlice - 1) / kSlice;
    const int64_t P = n_params(h1, h2, k);
    float* part = nullptr;
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&part),
                                  sizeof(float) * ((size_t)parts * P + parts), s));
    const size_t smem = sizeof(TrainSmem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) {
        k_mlp_loss_grad<<<parts, kMT, smem, s>>>(params, h1, h2, k, z, labels, q, n, part,
                                                 part + (size_t)parts * P);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_mlp_reduce<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(part, part + (size_t)parts * P,
                                                                 parts, P, n, grad, loss);
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(part, s);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return cuda_fail(e, "spmv_mlp_loss_grad");
    return SPMV_OK;
}
}  // namespace

spmv_status spmv_mlp_loss_grad(const float* params, int32_t h1, int32_t h2, int32_t k,
                               const float* z, const int32_t* labels, int32_t n, float* grad,
                               float* loss, spmv_stream_t stream)
{
    if (!labels) {
        clear_error();
        return fail(SPMV_ERR_INVALID_ARG, "spmv_mlp_loss_grad: NULL argument");
    }
    return loss_grad_impl(params, h1, h2, k, z, labels, nullptr, n, grad, loss, stream);
}

spmv_status spmv_mlp_loss_grad_soft(const float* params, int32_t h1, int32_t h2, int32_t k,
                                    const float* z, const float* q, int32_t n, float* grad,
                                    float* loss, spmv_stream_t stream)
{
    if (!q) {
        clear_error();
        return fail(SPMV_ERR_INVALID_ARG, "spmv_mlp_loss_grad_soft: NULL argument");
    }
    return loss_grad_impl(params, h1, h2, k, z, nullptr, q, n, grad, loss, stream);
}

spmv_status spmv_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t n,
                          int32_t step, float lr, float beta1, float beta2, float eps,
                          float weight_decay, spmv_stream_t stream)
{
    clear_error();
    if (!params || !grad || !m || !v || n < 0 || step < 1)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_mlp_adam: bad argument");
    if (n == 0) return SPMV_OK;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, grad, m, v, n, lr, beta1, beta2, eps,
                                                       weight_decay, c1, c2);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

}  // extern "C"
