// surr_api.cu -- C ABI of the surrogate MLP (include/surrogate.h): handle,
// parameters and statistics, training steps and rollouts.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "surr_kernels.cuh"
#include "surrogate.h"

static_assert(SURR_NPARAM == sg::NPARAM, "parameter count");
static_assert(SURR_NSTATS == sg::NSTATS, "statistics count");

struct surr_handle {
    surr_config cfg;
    ds::Phys phys;
    int device = 0, num_sms = 0, B = 0, splits = 0, stat_blocks = 0;
    long long step = 0;
    float *d_P = nullptr, *d_m = nullptr, *d_v = nullptr, *d_bias = nullptr, *d_stats = nullptr;
    uint8_t *d_imgA = nullptr, *d_imgW2 = nullptr, *d_imgB = nullptr, *d_imgW2T = nullptr;
    float *d_z1 = nullptr, *d_z2 = nullptr, *d_dy = nullptr, *d_db = nullptr, *d_loss_part = nullptr,
          *d_wpart = nullptr;
    uint8_t *d_xT = nullptr, *d_h1T = nullptr, *d_h2T = nullptr, *d_dz3T = nullptr, *d_dz2T = nullptr,
            *d_dz1T = nullptr;
    double* d_stat_part = nullptr;
    int* d_status = nullptr;
    cudaStream_t last = nullptr;
};

namespace {

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return SIM_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA;
}

#define SCK(x)                               \
    do {                                     \
        int r_ = cuda_rc(x);                 \
        if (r_) return r_;                   \
    } while (0)

template <class T>
int salloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) return SIM_OK;
    return cuda_rc(cudaMalloc((void**)p, n * sizeof(T)));
}

template <class T>
void sfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

bool fin_pos(float x) { return std::isfinite(x) && x > 0.f; }

int validate(const surr_config* c, const sim_config* p) {
    if (c->batch < 128 || c->batch > 262144 || c->batch % 128) return SIM_ERR_SIZE;
    if (c->splits < 0 || c->splits > 256) return SIM_ERR_INVALID_ARG;
    if (!fin_pos(c->lr) || !(c->beta1 >= 0.f && c->beta1 < 1.f) || !(c->beta2 >= 0.f && c->beta2 < 1.f) ||
        !fin_pos(c->eps) || !(c->margin >= 0.f && std::isfinite(c->margin)))
        return SIM_ERR_INVALID_ARG;
    for (int i = 0; i < 5; ++i)
        if (c->reserved[i]) return SIM_ERR_INVALID_ARG;
    if (p->model != SIM_MODEL_RIGID) return SIM_ERR_UNSUPPORTED;
    if (!fin_pos(p->dt) || !std::isfinite(p->gravity) || !fin_pos(p->mass)) return SIM_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        if (!fin_pos(p->inertia[i]) || !std::isfinite(p->k_rate[i]) || !std::isfinite(p->drag_body[i]) ||
            !std::isfinite(p->rate_scale[i]))
            return SIM_ERR_INVALID_ARG;
    return SIM_OK;
}

ds::Phys phys_of(const sim_config& c) {
    ds::Phys p;
    memset(&p, 0, sizeof(p));
    p.model = SIM_MODEL_RIGID; p.M = 1; p.D = 13; p.A = 4;
    p.dt = c.dt; p.g = c.gravity; p.mass = c.mass;
    for (int i = 0; i < 3; ++i) {
        p.J[i] = c.inertia[i]; p.K[i] = c.k_rate[i]; p.Dd[i] = c.drag_body[i]; p.rs[i] = c.rate_scale[i];
    }
    return p;
}

sg::SurrArgs fwd_args(const surr_handle* h) {
    sg::SurrArgs a;
    memset(&a, 0, sizeof(a));
    a.imgA = h->d_imgA; a.imgW2 = h->d_imgW2; a.bias = h->d_bias; a.stats = h->d_stats;
    a.c = h->phys; a.margin = h->cfg.margin; a.status = h->d_status;
    return a;
}

}  // namespace

extern "C" {

int surr_destroy(surr_handle* h) {
    if (!h) return SIM_OK;
    cudaDeviceSynchronize();
    sfree(h->d_P); sfree(h->d_m); sfree(h->d_v); sfree(h->d_bias); sfree(h->d_stats);
    sfree(h->d_imgA); sfree(h->d_imgW2); sfree(h->d_imgB); sfree(h->d_imgW2T);
    sfree(h->d_z1); sfree(h->d_z2); sfree(h->d_dy); sfree(h->d_db); sfree(h->d_loss_part); sfree(h->d_wpart);
    sfree(h->d_xT); sfree(h->d_h1T); sfree(h->d_h2T); sfree(h->d_dz3T); sfree(h->d_dz2T); sfree(h->d_dz1T);
    sfree(h->d_stat_part); sfree(h->d_status);
    delete h;
    return SIM_OK;
}

int surr_create(const surr_config* cfg, const sim_config* phys, surr_handle** out) {
    if (!cfg || !phys || !out) return SIM_ERR_NULL_PTR;
    *out = nullptr;
    int rc = validate(cfg, phys);
    if (rc) return rc;
    surr_handle* h = new (std::nothrow) surr_handle();
    if (!h) return SIM_ERR_OOM;
    h->cfg = *cfg;
    h->phys = phys_of(*phys);
    h->B = cfg->batch;
#define TRY(x)                \
    do {                      \
        int r_ = (x);         \
        if (r_) {             \
            surr_destroy(h);  \
            return r_;        \
        }                     \
    } while (0)
    TRY(cuda_rc(cudaGetDevice(&h->device)));
    TRY(cuda_rc(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)));
    const int nkb = h->B / 64;
    h->splits = cfg->splits ? cfg->splits : std::max(1, std::min(nkb, h->num_sms / 6));
    h->stat_blocks = 4 * h->num_sms;
    const size_t B = h->B;
    TRY(salloc(&h->d_P, sg::NPARAM)); TRY(salloc(&h->d_m, sg::NPARAM)); TRY(salloc(&h->d_v, sg::NPARAM));
    TRY(salloc(&h->d_bias, sg::NBIAS)); TRY(salloc(&h->d_stats, sg::NSTATS));
    TRY(salloc(&h->d_imgA, sg::IMG_A)); TRY(salloc(&h->d_imgW2, sg::IMG_W2));
    TRY(salloc(&h->d_imgB, sg::IMG_A)); TRY(salloc(&h->d_imgW2T, sg::IMG_W2));
    TRY(salloc(&h->d_z1, B * 256)); TRY(salloc(&h->d_z2, B * 256)); TRY(salloc(&h->d_dy, B * 16));
    TRY(salloc(&h->d_db, (B / 128) * 4 * sg::NBIAS)); TRY(salloc(&h->d_loss_part, B / 128));
    TRY(salloc(&h->d_wpart, (size_t)h->splits * 256 * (32 + 256 + 16)));
    TRY(salloc(&h->d_xT, 32 * B * 2)); TRY(salloc(&h->d_h1T, 256 * B * 2)); TRY(salloc(&h->d_h2T, 256 * B * 2));
    TRY(salloc(&h->d_dz3T, 16 * B * 2)); TRY(salloc(&h->d_dz2T, 256 * B * 2)); TRY(salloc(&h->d_dz1T, 256 * B * 2));
    TRY(salloc(&h->d_stat_part, (size_t)h->stat_blocks * 30 * 4));
    TRY(salloc(&h->d_status, 1));
    TRY(cuda_rc(cudaMemset(h->d_status, 0, sizeof(int))));
    std::vector<float> zero(sg::NPARAM, 0.f);
    *out = h;
    rc = surr_set_params(h, zero.data());
    if (rc) {
        *out = nullptr;
        surr_destroy(h);
        return rc;
    }
    std::vector<float> st(sg::NSTATS, 0.f);
    for (int k = 0; k < 17; ++k) {
        st[sg::ST_RSX + k] = 1.f;
        st[sg::ST_LOX + k] = -INFINITY;
        st[sg::ST_HIX + k] = INFINITY;
    }
    for (int k = 0; k < 13; ++k) st[sg::ST_SDD + k] = st[sg::ST_RSD + k] = 1.f;
    rc = surr_set_stats(h, st.data());
    if (rc) {
        *out = nullptr;
        surr_destroy(h);
        return rc;
    }
#undef TRY
    return SIM_OK;
}

int surr_set_params(surr_handle* h, const float* params) {
    if (!h || !params) return SIM_ERR_NULL_PTR;
    for (int i = 0; i < sg::NPARAM; ++i)
        if (!std::isfinite(params[i])) return SIM_ERR_INVALID_ARG;
    SCK(cudaMemcpy(h->d_P, params, sg::NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    SCK(cudaMemset(h->d_m, 0, sg::NPARAM * sizeof(float)));
    SCK(cudaMemset(h->d_v, 0, sg::NPARAM * sizeof(float)));
    h->step = 0;
    SCK(sg::launch_surr_pack(h->d_P, h->d_imgA, h->d_imgW2, h->d_imgB, h->d_imgW2T, h->d_bias, nullptr));
    SCK(cudaStreamSynchronize(nullptr));
    return SIM_OK;
}

int surr_get_params(surr_handle* h, float* params) {
    if (!h || !params) return SIM_ERR_NULL_PTR;
    SCK(cudaDeviceSynchronize());
    SCK(cudaMemcpy(params, h->d_P, sg::NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return SIM_OK;
}

int surr_set_stats(surr_handle* h, const float* stats) {
    if (!h || !stats) return SIM_ERR_NULL_PTR;
    for (int i = 0; i < sg::NSTATS; ++i)
        if (std::isnan(stats[i])) return SIM_ERR_INVALID_ARG;
    SCK(cudaMemcpy(h->d_stats, stats, sg::NSTATS * sizeof(float), cudaMemcpyHostToDevice));
    return SIM_OK;
}

int surr_get_stats(surr_handle* h, float* stats) {
    if (!h || !stats) return SIM_ERR_NULL_PTR;
    SCK(cudaDeviceSynchronize());
    SCK(cudaMemcpy(stats, h->d_stats, sg::NSTATS * sizeof(float), cudaMemcpyDeviceToHost));
    return SIM_OK;
}

int surr_fit_stats(surr_handle* h, const float* X, const float* S1, int64_t n, sim_stream_t stream) {
    if (!h || !X || !S1) return SIM_ERR_NULL_PTR;
    if (n < 1) return SIM_ERR_SIZE;
    h->last = (cudaStream_t)stream;
    SCK(sg::launch_surr_stats(X, S1, n, h->d_stat_part, h->stat_blocks, h->d_stats, h->last));
    return SIM_OK;
}

int surr_forward(surr_handle* h, const float* X, int64_t n, float* Y, sim_stream_t stream) {
    if (!h || !X || !Y) return SIM_ERR_NULL_PTR;
    if (n < 0 || n > INT32_MAX - 128) return SIM_ERR_SIZE;
    if (n == 0) return SIM_OK;
    sg::SurrArgs a = fwd_args(h);
    a.mode = 1;
    a.N = (int)n;
    a.T = 1;
    a.X = X;
    a.Y = Y;
    h->last = (cudaStream_t)stream;
    SCK(sg::launch_surr_fwd(a, h->num_sms, h->last));
    return SIM_OK;
}

int surr_rollout(surr_handle* h, const float* s0, const float* actions, int32_t N, int32_t T, float* states,
                 float* sT, uint8_t* fallback, sim_stream_t stream) {
    if (!h || !s0 || !actions) return SIM_ERR_NULL_PTR;
    if (N < 0 || T < 0 || (int64_t)N > INT32_MAX - 128) return SIM_ERR_SIZE;
    if (N == 0) return SIM_OK;
    sg::SurrArgs a = fwd_args(h);
    a.mode = 0;
    a.N = N;
    a.T = T;
    a.s0 = s0;
    a.actions = actions;
    a.states = states;
    a.sT = sT;
    a.fallback = fallback;
    h->last = (cudaStream_t)stream;
    SCK(sg::launch_surr_fwd(a, h->num_sms, h->last));
    return SIM_OK;
}

int surr_train_step(surr_handle* h, const float* X, const float* S1, const int32_t* idx, float* loss,
                    float* grads, int32_t apply, sim_stream_t stream) {
    if (!h || !X || !S1 || !idx) return SIM_ERR_NULL_PTR;
    sg::TrainArgs a;
    memset(&a, 0, sizeof(a));
    a.imgA = h->d_imgA; a.imgW2 = h->d_imgW2; a.imgB = h->d_imgB; a.imgW2T = h->d_imgW2T;
    a.bias = h->d_bias; a.stats = h->d_stats;
    a.X = X; a.S1 = S1; a.idx = idx; a.B = h->B;
    a.z1 = h->d_z1; a.z2 = h->d_z2; a.dy = h->d_dy;
    a.xT = h->d_xT; a.h1T = h->d_h1T; a.h2T = h->d_h2T; a.dz3T = h->d_dz3T; a.dz2T = h->d_dz2T; a.dz1T = h->d_dz1T;
    a.db_part = h->d_db; a.loss_part = h->d_loss_part; a.wpart = h->d_wpart; a.splits = h->splits;
    a.P = h->d_P; a.m = h->d_m; a.v = h->d_v; a.grads = grads; a.loss = loss;
    a.lr = h->cfg.lr; a.beta1 = h->cfg.beta1; a.beta2 = h->cfg.beta2; a.eps = h->cfg.eps;
    a.apply = apply ? 1 : 0;
    const long long step = h->step + (apply ? 1 : 0);
    a.c1 = step > 0 ? (float)(1.0 / (1.0 - std::pow((double)h->cfg.beta1, (double)step))) : 1.f;
    a.c2 = step > 0 ? (float)(1.0 / (1.0 - std::pow((double)h->cfg.beta2, (double)step))) : 1.f;
    a.status = h->d_status;
    h->last = (cudaStream_t)stream;
    SCK(sg::launch_surr_train(a, h->last));
    h->step = step;
    return SIM_OK;
}

int surr_last_status(surr_handle* h, int32_t* status) {
    if (!h || !status) return SIM_ERR_NULL_PTR;
    SCK(cudaStreamSynchronize(h->last));
    int v = 0;
    SCK(cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    SCK(cudaMemset(h->d_status, 0, sizeof(int)));
    *status = v;
    if (v & SIM_STATUS_TIMEOUT) return SIM_ERR_TIMEOUT;
    if (v & SIM_STATUS_NAN) return SIM_ERR_NAN;
    return SIM_OK;
}

}  // extern "C"
