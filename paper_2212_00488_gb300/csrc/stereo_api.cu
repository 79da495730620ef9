// C ABI of the library (include/stereo.h): context, workspace, argument
// checks and the order of the pipeline's kernels (Sec. III steps 1-8).
#include "../../include/stereo.h"
#include "internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

using namespace stereo;

struct stereo_ctx {
    int device = 0;
    stereo_params p{};
    size_t mem_cap = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    uint32_t lut_host[256 + 8];     // quantised AD costs [256], then census costs [8]
    uint32_t P = 0;
    uint32_t *d_lut = nullptr;
    uint32_t *d_err = nullptr;      // device error word of the fused kernel's bounded waits
    uint32_t *h_err = nullptr;      // pinned host copy
    uint32_t wait_limit = 1u << 20;

    void *ws = nullptr;
    size_t ws_size = 0;

    // layout of the current frame inside ws
    int W = 0, H = 0, Dmax = 0, X = 0, Y = 0, D = 0;
    bool host_staging = false;
    uint8_t *gf[2] = {nullptr, nullptr};   // full-res grey (the processed grey without downscaling)
    uint8_t *gs[2] = {nullptr, nullptr};   // processed grey
    uint32_t *pix[2] = {nullptr, nullptr};
    uint32_t *arm[2] = {nullptr, nullptr};
    uint32_t *armc[2] = {nullptr, nullptr};   // [Y + wy][X] arm words of the fused kernel
    uint32_t *key[2] = {nullptr, nullptr};
    uint8_t *dm = nullptr;
    float *dplus_ws = nullptr;
    uint8_t *stage_rgb[2] = {nullptr, nullptr};
    float *stage_disp = nullptr;
    uint8_t *stage_maps = nullptr;

    // the last compute, for stereo_launch_stage / stereo_debug_planes
    bool have_frame = false;
    const uint8_t *in_l = nullptr, *in_r = nullptr;
    float *out_disp = nullptr, *dplus = nullptr;
    uint8_t *out_dl = nullptr, *out_dr = nullptr, *out_gcp = nullptr;
    int launches = 0;
    int tile = -1;          // fused-kernel tile shape, -1 = automatic
    int num_sms = 0;

    // Profiling: a ring of event sets, one per recent frame, harvested when a
    // slot is reused (by then its frame has long finished), so timing adds no
    // synchronisation to a stream of back-to-back frames.
    struct ProfSlot {
        cudaEvent_t ev[STEREO_NUM_STAGES + 1] = {};
        bool ran[STEREO_NUM_STAGES] = {};
        bool pending = false;
    };
    static constexpr int kProfRing = 64;
    bool prof = false;
    int prof_period = 1;                      // profile every prof_period-th compute
    long prof_count = 0;
    bool prof_events = false;
    ProfSlot prof_ring[kProfRing];
    int prof_next = 0;
    double prof_acc[STEREO_NUM_STAGES] = {};
    int prof_n = 0;

    // Batched frames: their own workspace, the graph of the last batch and
    // the autotuner's choices of tile shape per batch signature.
    void *bws = nullptr;
    size_t bws_size = 0;
    std::map<int, cudaGraphExec_t> bexec;   // one graph per batch size, updated in place
    cudaGraphExec_t dexec[2] = {nullptr, nullptr};   // differentiable forward / backward graphs
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    std::map<std::string, int> tune;
    void *dws = nullptr;            // workspace of the differentiable form
    size_t dws_size = 0;
    int last_batch_tile = -1;
    float last_batch_tune_ms[kNumTiles] = {};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(stereo_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(stereo_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, STEREO_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Eqs. 4-5 on intensities scaled to [0, 1], quantised to round(scale * v),
// half away from zero, evaluated in double on the host; the device only reads
// the tables. AD by |grey difference| (0..255), census by Hamming distance
// (0..6; entry 7 never occurs).
void build_lut(stereo_ctx *c)
{
    const double s = c->p.cost_scale;
    uint32_t *ad = c->lut_host, *mc = c->lut_host + 256;
    for (int a = 0; a < 256; ++a)
        ad[a] = (uint32_t)std::llround(s * (1.0 - std::exp(-((double)a / 255.0) / c->p.lambda_ad)));
    for (int h = 0; h <= 6; ++h)
        mc[h] = (uint32_t)std::llround(s * (1.0 - std::exp(-(double)h / c->p.lambda_mc)));
    mc[7] = mc[6];
    c->P = ad[255] + mc[6];
}

int check_params(stereo_ctx *c, const stereo_params &p)
{
    if (!(p.lambda_ad > 0) || !(p.lambda_mc > 0)) return fail(c, STEREO_EINVAL, "lambda_ad and lambda_mc must be > 0");
    if (p.tc < 0 || p.tc > 256) return fail(c, STEREO_EINVAL, "tc must be in [0, 256]");
    if (p.wx < 0 || p.wx > kMaxWx) return fail(c, STEREO_EINVAL, "wx must be in [0, %d]", kMaxWx);
    if (p.wy < 0 || p.wy > kMaxWy) return fail(c, STEREO_EINVAL, "wy must be in [0, %d]", kMaxWy);
    if (p.t_fill < 0 || p.t_fill > 255) return fail(c, STEREO_EINVAL, "t_fill must be in [0, 255]");
    if (p.downscale != 0 && p.downscale != 1) return fail(c, STEREO_EINVAL, "downscale must be 0 or 1");
    if (p.fill_mode < 0 || p.fill_mode > 2) return fail(c, STEREO_EINVAL, "fill_mode must be 0, 1 or 2");
    if (p.cost_scale < 1 || p.cost_scale > (1 << 20)) return fail(c, STEREO_EINVAL, "cost_scale must be in [1, 2^20]");
    // the fused kernel keeps the cost table in 16 bits
    if (p.cost_scale * ((1.0 - std::exp(-1.0 / p.lambda_ad)) + (1.0 - std::exp(-6.0 / p.lambda_mc))) + 1.0 > 65535.0)
        return fail(c, STEREO_EINVAL, "cost_scale %d too large: a matching cost must stay below 2^16", p.cost_scale);
    // the packed WTA key holds the aggregated cost in 24 bits
    const double pmax = p.cost_scale * ((1.0 - std::exp(-1.0 / p.lambda_ad)) + (1.0 - std::exp(-6.0 / p.lambda_mc))) + 1.0;
    const double worst = (double)(2 * p.wx + 1) * (2 * p.wy + 1) * pmax;
    if (worst >= 16777216.0)
        return fail(c, STEREO_EINVAL, "cost_scale %d too large for wx=%d wy=%d: an aggregated cost could reach 2^24",
                    p.cost_scale, p.wx, p.wy);
    return STEREO_OK;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// Lays out (or only measures, when base is null) the workspace of one frame.
size_t layout(stereo_ctx *c, char *base, int W, int H, bool staging)
{
    const bool ds = c->p.downscale != 0;
    const int X = ds ? W / 2 : W, Y = ds ? H / 2 : H;
    const size_t nf = (size_t)W * H, nl = (size_t)X * Y;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    for (int i = 0; i < 2; ++i) c->gf[i] = (uint8_t *)take(nf);
    for (int i = 0; i < 2; ++i) c->gs[i] = ds ? (uint8_t *)take(nl) : c->gf[i];
    for (int i = 0; i < 2; ++i) c->pix[i] = (uint32_t *)take(nl * 4);
    for (int i = 0; i < 2; ++i) c->arm[i] = (uint32_t *)take(nl * 4);
    for (int i = 0; i < 2; ++i) c->armc[i] = (uint32_t *)take(armc_words(X, Y, c->p.wy) * 4);
    for (int i = 0; i < 2; ++i) c->key[i] = (uint32_t *)take(nl * 4);
    c->dm = (uint8_t *)take(nl);
    c->dplus_ws = (float *)take(nl * 4);
    if (staging) {
        for (int i = 0; i < 2; ++i) c->stage_rgb[i] = (uint8_t *)take(nf * 3);
        c->stage_disp = (float *)take(nf * 4);
        c->stage_maps = (uint8_t *)take(nl * 3);
    } else {
        c->stage_rgb[0] = c->stage_rgb[1] = nullptr;
        c->stage_disp = nullptr;
        c->stage_maps = nullptr;
    }
    return off;
}

int ensure_workspace(stereo_ctx *c, int W, int H, int Dmax, bool staging)
{
    const size_t need = layout(c, nullptr, W, H, staging);
    if (need > c->ws_size) {
        if (c->mem_cap && need > c->mem_cap)
            return fail(c, STEREO_ENOMEM, "workspace of %zu bytes exceeds the cap of %zu", need, c->mem_cap);
        if (c->ws) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->ws);
            c->ws = nullptr;
            c->ws_size = 0;
        }
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, STEREO_ENOMEM, "cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
        }
        c->ws = p;
        c->ws_size = need;
    }
    layout(c, (char *)c->ws, W, H, staging);
    c->W = W;
    c->H = H;
    c->Dmax = Dmax;
    c->X = c->p.downscale ? W / 2 : W;
    c->Y = c->p.downscale ? H / 2 : H;
    c->D = c->p.downscale ? (Dmax + 1) / 2 : Dmax;
    c->host_staging = staging;
    return STEREO_OK;
}

int check_frame(stereo_ctx *c, const void *l, const void *r, int W, int H, int Dmax, const float *disp)
{
    if (!l || !r || !disp) return fail(c, STEREO_EINVAL, "left, right and disp_out must not be NULL");
    if (W < 1 || H < 1 || W > 8192 || H > 8192) return fail(c, STEREO_EINVAL, "W and H must be in [1, 8192]");
    if (c->p.downscale && (W < 2 || H < 2)) return fail(c, STEREO_EINVAL, "downscaling needs W, H >= 2");
    const int D = c->p.downscale ? (Dmax + 1) / 2 : Dmax;
    if (Dmax < 1 || D > 256) return fail(c, STEREO_EINVAL, "Dmax %d out of range (at most 256 processed disparities)", Dmax);
    const int X = c->p.downscale ? W / 2 : W;
    if (X > 4096) return fail(c, STEREO_EINVAL, "processed width %d exceeds 4096", X);
    return STEREO_OK;
}

// Launches one stage of the current frame on stream s.
cudaError_t run_stage(stereo_ctx *c, int stage, cudaStream_t s)
{
    const bool ds = c->p.downscale != 0;
    switch (stage) {
    case STEREO_STAGE_SCALEDOWN: {
        if (ds)
            return launch_grey_down(c->in_l, c->in_r, c->gf[0], c->gf[1], c->gs[0], c->gs[1], c->W, c->H, s,
                                    &c->launches);
        c->launches++;
        return launch_grey(c->in_l, c->in_r, c->gf[0], c->gf[1], c->W, c->H, s);
    }
    case STEREO_STAGE_SUPPORT:
        c->launches++;
        return launch_support(c->gs[0], c->gs[1], c->pix[0], c->pix[1], c->arm[0], c->arm[1], c->armc[0],
                              c->armc[1], c->key[0], c->key[1], c->d_err, c->X, c->Y, c->p.wx, c->p.wy,
                              c->p.tc, s);
    case STEREO_STAGE_COSTAGG: {
        CostAggArgs a;
        a.pix_l = c->pix[0];
        a.pix_r = c->pix[1];
        a.arm_l = c->arm[0];
        a.arm_r = c->arm[1];
        a.armc_l = c->armc[0];
        a.armc_r = c->armc[1];
        a.key_l = c->key[0];
        a.key_r = c->key[1];
        a.lut_ad = c->d_lut;
        a.lut_mc = c->d_lut + 256;
        a.err = c->d_err;
        a.wait_limit = c->wait_limit;
        a.X = c->X;
        a.Y = c->Y;
        a.D = c->D;
        a.wx = c->p.wx;
        a.wy = c->p.wy;
        a.P = c->P;
        a.tile = c->tile;
        a.num_sms = c->num_sms;
        c->launches++;
        return launch_costagg(a, s);
    }
    case STEREO_STAGE_REFINE:
        c->launches++;
        if (ds)   // the scale-up runs in the same kernel
            return launch_refine_up(c->key[0], c->key[1], c->gs[0], c->gf[0], c->X, c->Y, c->W, c->H, c->p.t_fill,
                                    c->p.fill_mode, c->out_dl, c->out_dr, c->out_gcp, c->dm, c->dplus, c->out_disp, s);
        return launch_refine(c->key[0], c->key[1], c->gs[0], c->X, c->Y, c->p.t_fill, c->p.fill_mode, c->out_dl, c->out_dr,
                             c->out_gcp, c->dm, c->dplus, s);
    case STEREO_STAGE_UPSCALE:
        return cudaSuccess;   // inside the refine stage's kernel (downscaling) or nothing to do
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t harvest(stereo_ctx *c, stereo_ctx::ProfSlot &sl)
{
    if (!sl.pending) return cudaSuccess;
    sl.pending = false;
    cudaError_t e = cudaEventSynchronize(sl.ev[STEREO_NUM_STAGES]);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < STEREO_NUM_STAGES; ++i) {
        if (!sl.ran[i]) continue;
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, sl.ev[i], sl.ev[i + 1])) != cudaSuccess) return e;
        c->prof_acc[i] += t;
    }
    c->prof_n++;
    return cudaSuccess;
}

int run_frame(stereo_ctx *c, cudaStream_t s)
{
    c->launches = 0;
    stereo_ctx::ProfSlot *sl = nullptr;
    if (c->prof && c->prof_count++ % c->prof_period == 0) {
        sl = &c->prof_ring[c->prof_next];
        c->prof_next = (c->prof_next + 1) % stereo_ctx::kProfRing;
        cudaError_t e = harvest(c, *sl);
        if (e != cudaSuccess) return cuda_fail(c, e, "profiling events");
    }
    for (int st = 0; st < STEREO_NUM_STAGES; ++st) {
        if (sl) cudaEventRecord(sl->ev[st], s);
        cudaError_t e = run_stage(c, st, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
        if (sl) sl->ran[st] = st != STEREO_STAGE_UPSCALE;
    }
    if (sl) {
        cudaEventRecord(sl->ev[STEREO_NUM_STAGES], s);
        sl->pending = true;
    }
    return STEREO_OK;
}

}  // namespace

extern "C" {

void stereo_default_params(stereo_params *out)
{
    if (!out) return;
    out->lambda_ad = 0.3;
    out->lambda_mc = 2.3;
    out->tc = 13;
    out->wx = 21;
    out->wy = 31;
    out->t_fill = 3;
    out->downscale = 1;
    out->cost_scale = 512;
    out->fill_mode = 0;
}

int stereo_create(stereo_ctx **out, int device, const stereo_params *p, size_t mem_cap_bytes)
{
    if (!out) return STEREO_EINVAL;
    *out = nullptr;
    stereo_ctx *c = new (std::nothrow) stereo_ctx();
    if (!c) return STEREO_ENOMEM;
    if (p) c->p = *p; else stereo_default_params(&c->p);
    int rc = check_params(c, c->p);
    if (rc != STEREO_OK) { delete c; return rc; }
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        delete c;
        return e != cudaSuccess ? STEREO_ECUDA : STEREO_EINVAL;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess || prop.major != 10 || prop.minor != 3) {
        cudaGetLastError();
        delete c;
        return STEREO_EINVAL;   // the kernels are built for sm_103a only
    }
    c->device = device;
    c->mem_cap = mem_cap_bytes;
    c->num_sms = prop.multiProcessorCount;
    DeviceGuard g(device);
    build_lut(c);
    if ((e = costagg_setup()) != cudaSuccess || (e = refine_setup()) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_lut, sizeof c->lut_host)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_lut, c->lut_host, sizeof c->lut_host, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_err, sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(c->d_err, 0, sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaHostAlloc(&c->h_err, sizeof(uint32_t), cudaHostAllocDefault)) != cudaSuccess) {
        cudaGetLastError();
        stereo_destroy(c);
        return STEREO_ECUDA;
    }
    for (cudaEvent_t *ev : {&c->ev_in, &c->ev_out})
        if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) {
            cudaGetLastError();
            stereo_destroy(c);
            return STEREO_ECUDA;
        }
    for (cudaEvent_t *ev : {&c->ev_t0, &c->ev_t1})
        if ((e = cudaEventCreate(ev)) != cudaSuccess) {
            cudaGetLastError();
            stereo_destroy(c);
            return STEREO_ECUDA;
        }
    *out = c;
    return STEREO_OK;
}

void stereo_destroy(stereo_ctx *c)
{
    if (!c) return;
    {
        DeviceGuard g(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        for (auto &sl : c->prof_ring)
            for (auto &ev : sl.ev)
                if (ev) cudaEventDestroy(ev);
        if (c->ws) cudaFree(c->ws);
        if (c->bws) cudaFree(c->bws);
        if (c->dws) cudaFree(c->dws);
        for (auto &kv : c->bexec) cudaGraphExecDestroy(kv.second);
        for (cudaGraphExec_t ge : c->dexec)
            if (ge) cudaGraphExecDestroy(ge);
        for (cudaEvent_t ev : {c->ev_in, c->ev_out, c->ev_t0, c->ev_t1})
            if (ev) cudaEventDestroy(ev);
        if (c->d_lut) cudaFree(c->d_lut);
        if (c->d_err) cudaFree(c->d_err);
        if (c->h_err) cudaFreeHost(c->h_err);
        if (c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
}

const char *stereo_last_error(const stereo_ctx *c)
{
    return c ? c->err.c_str() : "null context";
}

int stereo_compute(stereo_ctx *c, const uint8_t *left_rgb, const uint8_t *right_rgb, int W, int H, int Dmax,
                   float *disp_out, uint8_t *dl_out, uint8_t *dr_out, uint8_t *gcp_out, void *stream)
{
    if (!c) return STEREO_EINVAL;
    c->err.clear();
    int rc = check_frame(c, left_rgb, right_rgb, W, H, Dmax, disp_out);
    if (rc != STEREO_OK) return rc;
    DeviceGuard g(c->device);
    rc = ensure_workspace(c, W, H, Dmax, c->host_staging);
    if (rc != STEREO_OK) return rc;
    c->in_l = left_rgb;
    c->in_r = right_rgb;
    c->out_disp = disp_out;
    c->out_dl = dl_out;
    c->out_dr = dr_out;
    c->out_gcp = gcp_out;
    c->dplus = c->p.downscale ? c->dplus_ws : disp_out;
    c->have_frame = true;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    return run_frame(c, s);
}

int stereo_compute_host_async(stereo_ctx *c, const uint8_t *left_rgb, const uint8_t *right_rgb, int W, int H,
                              int Dmax, float *disp_out, uint8_t *dl_out, uint8_t *dr_out, uint8_t *gcp_out)
{
    if (!c) return STEREO_EINVAL;
    c->err.clear();
    int rc = check_frame(c, left_rgb, right_rgb, W, H, Dmax, disp_out);
    if (rc != STEREO_OK) return rc;
    DeviceGuard g(c->device);
    rc = ensure_workspace(c, W, H, Dmax, true);
    if (rc != STEREO_OK) return rc;
    cudaStream_t s = c->stream;
    const size_t nf = (size_t)W * H, nl = (size_t)c->X * c->Y;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->stage_rgb[0], left_rgb, nf * 3, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->stage_rgb[1], right_rgb, nf * 3, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(c, e, "host-to-device copy");
    c->in_l = c->stage_rgb[0];
    c->in_r = c->stage_rgb[1];
    c->out_disp = c->stage_disp;
    c->out_dl = dl_out ? c->stage_maps : nullptr;
    c->out_dr = dr_out ? c->stage_maps + nl : nullptr;
    c->out_gcp = gcp_out ? c->stage_maps + 2 * nl : nullptr;
    c->dplus = c->p.downscale ? c->dplus_ws : c->stage_disp;
    c->have_frame = true;
    rc = run_frame(c, s);
    if (rc != STEREO_OK) return rc;
    if ((e = cudaMemcpyAsync(disp_out, c->stage_disp, nf * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(c, e, "device-to-host copy");
    if (dl_out && (e = cudaMemcpyAsync(dl_out, c->stage_maps, nl, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(c, e, "device-to-host copy");
    if (dr_out && (e = cudaMemcpyAsync(dr_out, c->stage_maps + nl, nl, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(c, e, "device-to-host copy");
    if (gcp_out && (e = cudaMemcpyAsync(gcp_out, c->stage_maps + 2 * nl, nl, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(c, e, "device-to-host copy");
    if ((e = cudaMemcpyAsync(c->h_err, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(c, e, "device-to-host copy");
    return STEREO_OK;
}

int stereo_compute_host(stereo_ctx *c, const uint8_t *left_rgb, const uint8_t *right_rgb, int W, int H,
                        int Dmax, float *disp_out, uint8_t *dl_out, uint8_t *dr_out, uint8_t *gcp_out)
{
    const int rc = stereo_compute_host_async(c, left_rgb, right_rgb, W, H, Dmax, disp_out, dl_out, dr_out, gcp_out);
    if (rc != STEREO_OK) return rc;
    DeviceGuard g(c->device);
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    if (*c->h_err) return fail(c, STEREO_ETIMEOUT, "a bounded wait in the fused kernel gave up");
    return STEREO_OK;
}

int stereo_sync(stereo_ctx *c)
{
    if (!c) return STEREO_EINVAL;
    DeviceGuard g(c->device);
    // the error word is read on the context's own stream, after its work
    cudaError_t e = cudaMemcpyAsync(c->h_err, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    if (*c->h_err) return fail(c, STEREO_ETIMEOUT, "a bounded wait in the fused kernel gave up");
    return STEREO_OK;
}

int stereo_set_wait_limit(stereo_ctx *c, uint32_t polls)
{
    if (!c) return STEREO_EINVAL;
    c->wait_limit = polls;
    return STEREO_OK;
}

int stereo_debug_planes(stereo_ctx *c, uint8_t *grey_l, uint8_t *grey_r, uint8_t *census_l, uint8_t *census_r,
                        uint32_t *arms_l, uint32_t *arms_r, uint8_t *dm, float *dplus, void *stream)
{
    if (!c) return STEREO_EINVAL;
    if (!c->have_frame) return fail(c, STEREO_EINVAL, "no frame has been computed");
    DeviceGuard g(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const size_t nl = (size_t)c->X * c->Y;
    cudaError_t e = launch_unpack_planes(c->pix[0], c->arm[0], grey_l, census_l, arms_l, c->X, c->Y, s);
    if (e == cudaSuccess) e = launch_unpack_planes(c->pix[1], c->arm[1], grey_r, census_r, arms_r, c->X, c->Y, s);
    if (e == cudaSuccess && dm) e = cudaMemcpyAsync(dm, c->dm, nl, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && dplus) e = cudaMemcpyAsync(dplus, c->dplus, nl * 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? STEREO_OK : cuda_fail(c, e, "debug planes");
}

int stereo_launch_stage(stereo_ctx *c, int stage, void *stream)
{
    if (!c) return STEREO_EINVAL;
    if (!c->have_frame) return fail(c, STEREO_EINVAL, "no frame has been computed");
    if (stage < 0 || stage >= STEREO_NUM_STAGES) return fail(c, STEREO_EINVAL, "stage %d out of range", stage);
    DeviceGuard g(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    cudaError_t e = run_stage(c, stage, s);
    return e == cudaSuccess ? STEREO_OK : cuda_fail(c, e, "kernel launch");
}

int stereo_set_profiling(stereo_ctx *c, int on)
{
    if (!c || on < 0) return STEREO_EINVAL;
    DeviceGuard g(c->device);
    if (on && !c->prof_events) {
        for (auto &sl : c->prof_ring)
            for (auto &ev : sl.ev) {
                cudaError_t e = cudaEventCreate(&ev);
                if (e != cudaSuccess) return cuda_fail(c, e, "event create");
            }
        c->prof_events = true;
    }
    for (auto &sl : c->prof_ring) {
        if (sl.pending) cudaEventSynchronize(sl.ev[STEREO_NUM_STAGES]);
        sl.pending = false;
    }
    for (double &a : c->prof_acc) a = 0.0;
    c->prof_n = 0;
    c->prof_next = 0;
    c->prof = on > 0;
    c->prof_period = on > 0 ? on : 1;
    c->prof_count = 0;
    return STEREO_OK;
}

int stereo_stage_ms(stereo_ctx *c, float *ms, int n)
{
    if (!c || !ms || n < 0 || n > STEREO_NUM_STAGES) return STEREO_EINVAL;
    DeviceGuard g(c->device);
    for (auto &sl : c->prof_ring) {
        cudaError_t e = harvest(c, sl);
        if (e != cudaSuccess) return cuda_fail(c, e, "profiling events");
    }
    if (c->prof_n == 0) return fail(c, STEREO_EINVAL, "no profiled compute since profiling was turned on");
    for (int i = 0; i < n; ++i) ms[i] = (float)(c->prof_acc[i] / c->prof_n);
    return c->prof_n;
}

int stereo_last_launch_count(const stereo_ctx *c)
{
    return c ? c->launches : 0;
}

int stereo_set_tile(stereo_ctx *c, int tile)
{
    if (!c) return STEREO_EINVAL;
    if (tile < -1 || tile >= kNumTiles) return fail(c, STEREO_EINVAL, "tile %d out of range [-1, %d]", tile, kNumTiles - 1);
    c->tile = tile;
    return STEREO_OK;
}

int stereo_get_tile(stereo_ctx *c, int W, int H, int Dmax)
{
    if (!c || W < 1 || H < 1 || Dmax < 1) return STEREO_EINVAL;
    if (c->tile >= 0) return c->tile;
    CostAggArgs a{};
    a.X = c->p.downscale ? W / 2 : W;
    a.Y = c->p.downscale ? H / 2 : H;
    a.D = c->p.downscale ? (Dmax + 1) / 2 : Dmax;
    a.wx = c->p.wx;
    a.wy = c->p.wy;
    a.P = c->P;
    return costagg_pick(a, c->num_sms);
}

}  // extern "C"

// ---------------------------------------------------------------- batches

namespace {

// Device workspace of one frame of a batch.
struct FrameWs {
    int W, H, Dmax, X, Y, D;
    uint8_t *gf[2], *gs[2];
    uint32_t *pix[2], *arm[2], *armc[2], *key[2];
    uint8_t *dm;
    float *dplus;
};

size_t frame_layout(const stereo_params &p, int W, int H, int Dmax, char *base, FrameWs *f)
{
    const bool ds = p.downscale != 0;
    const int X = ds ? W / 2 : W, Y = ds ? H / 2 : H;
    const size_t nf = (size_t)W * H, nl = (size_t)X * Y;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *q = base ? base + off : nullptr;
        off += align256(bytes);
        return q;
    };
    FrameWs g{};
    g.W = W;
    g.H = H;
    g.Dmax = Dmax;
    g.X = X;
    g.Y = Y;
    g.D = ds ? (Dmax + 1) / 2 : Dmax;
    for (int i = 0; i < 2; ++i) g.gf[i] = (uint8_t *)take(nf);
    for (int i = 0; i < 2; ++i) g.gs[i] = ds ? (uint8_t *)take(nl) : g.gf[i];
    for (int i = 0; i < 2; ++i) g.pix[i] = (uint32_t *)take(nl * 4);
    for (int i = 0; i < 2; ++i) g.arm[i] = (uint32_t *)take(nl * 4);
    for (int i = 0; i < 2; ++i) g.armc[i] = (uint32_t *)take(armc_words(X, Y, p.wy) * 4);
    for (int i = 0; i < 2; ++i) g.key[i] = (uint32_t *)take(nl * 4);
    g.dm = (uint8_t *)take(nl);
    g.dplus = (float *)take(nl * 4);
    if (f) *f = g;
    return off;
}

CostAggArgs frame_args(const stereo_ctx *c, const FrameWs &f)
{
    CostAggArgs a{};
    a.pix_l = f.pix[0];
    a.pix_r = f.pix[1];
    a.arm_l = f.arm[0];
    a.arm_r = f.arm[1];
    a.armc_l = f.armc[0];
    a.armc_r = f.armc[1];
    a.key_l = f.key[0];
    a.key_r = f.key[1];
    a.lut_ad = c->d_lut;
    a.lut_mc = c->d_lut + 256;
    a.err = c->d_err;
    a.wait_limit = c->wait_limit;
    a.X = f.X;
    a.Y = f.Y;
    a.D = f.D;
    a.wx = c->p.wx;
    a.wy = c->p.wy;
    a.P = c->P;
    a.tile = -1;
    a.num_sms = c->num_sms;
    return a;
}

cudaError_t batch_prep(stereo_ctx *c, const stereo_job &j, const FrameWs &f, cudaStream_t s, int &launches)
{
    cudaError_t e;
    if (c->p.downscale) {
        e = launch_grey_down(j.left_rgb, j.right_rgb, f.gf[0], f.gf[1], f.gs[0], f.gs[1], f.W, f.H, s, &launches);
    } else {
        e = launch_grey(j.left_rgb, j.right_rgb, f.gf[0], f.gf[1], f.W, f.H, s);
        launches++;
    }
    if (e == cudaSuccess) {
        e = launch_support(f.gs[0], f.gs[1], f.pix[0], f.pix[1], f.arm[0], f.arm[1], f.armc[0], f.armc[1],
                           f.key[0], f.key[1], c->d_err, f.X, f.Y, c->p.wx, c->p.wy, c->p.tc, s);
        launches++;
    }
    return e;
}

cudaError_t batch_post(stereo_ctx *c, const stereo_job &j, const FrameWs &f, cudaStream_t s, int &launches)
{
    launches++;
    if (c->p.downscale)
        return launch_refine_up(f.key[0], f.key[1], f.gs[0], f.gf[0], f.X, f.Y, f.W, f.H, c->p.t_fill, c->p.fill_mode,
                                j.dl_out, j.dr_out, j.gcp_out, f.dm, f.dplus, j.disp_out, s);
    return launch_refine(f.key[0], f.key[1], f.gs[0], f.X, f.Y, c->p.t_fill, c->p.fill_mode, j.dl_out, j.dr_out,
                         j.gcp_out, f.dm, j.disp_out, s);
}

std::string batch_signature(const stereo_ctx *c, const std::vector<FrameWs> &fw)
{
    char buf[512];
    cudaDeviceProp prop;
    const char *name = cudaGetDeviceProperties(&prop, c->device) == cudaSuccess ? prop.name : "gpu";
    snprintf(buf, sizeof buf, "%.200s sms%d wx%d wy%d scale%d ds%d |", name, c->num_sms, c->p.wx, c->p.wy,
             c->p.cost_scale, c->p.downscale);
    std::string sig = buf;
    std::vector<std::string> parts;
    for (const FrameWs &f : fw) {
        snprintf(buf, sizeof buf, " %dx%dx%d", f.X, f.Y, f.D);
        parts.push_back(buf);
    }
    std::sort(parts.begin(), parts.end());
    for (const std::string &q : parts) sig += q;
    for (char &ch : sig)
        if (ch == '\t' || ch == '\n') ch = ' ';
    return sig;
}

}  // namespace

extern "C" {

int stereo_compute_batch(stereo_ctx *c, int n, const stereo_job *jobs, void *stream)
{
    if (!c) return STEREO_EINVAL;
    c->err.clear();
    if (n < 1 || n > kMaxBatch || !jobs) return fail(c, STEREO_EINVAL, "batch size must be in [1, %d]", kMaxBatch);
    for (int i = 0; i < n; ++i) {
        int rc = check_frame(c, jobs[i].left_rgb, jobs[i].right_rgb, jobs[i].W, jobs[i].H, jobs[i].Dmax,
                             jobs[i].disp_out);
        if (rc != STEREO_OK) return fail(c, rc, "job %d: %s", i, c->err.c_str());
    }
    DeviceGuard g(c->device);

    // jobs largest first, so the persistent kernel starts the long sweeps early
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto work = [&](int i) {
        const stereo_job &j = jobs[i];
        const double X = c->p.downscale ? j.W / 2 : j.W, Y = c->p.downscale ? j.H / 2 : j.H;
        const double D = c->p.downscale ? (j.Dmax + 1) / 2 : j.Dmax;
        return X * Y * D;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });

    // workspace: one frame layout per job plus the tile counter
    std::vector<size_t> offs(n);
    size_t need = 256;
    for (int k = 0; k < n; ++k) {
        const stereo_job &j = jobs[order[k]];
        offs[k] = need;
        need += frame_layout(c->p, j.W, j.H, j.Dmax, nullptr, nullptr);
    }
    if (need > c->bws_size) {
        if (c->mem_cap && need + c->ws_size > c->mem_cap)
            return fail(c, STEREO_ENOMEM, "batch workspace of %zu bytes exceeds the cap", need);
        if (c->bws) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->bws);
            c->bws = nullptr;
            c->bws_size = 0;
        }
        if (cudaMalloc(&c->bws, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, STEREO_ENOMEM, "cudaMalloc(%zu) for the batch failed", need);
        }
        c->bws_size = need;
    }
    std::vector<FrameWs> fw(n);
    BatchArgs b{};
    b.njobs = n;
    b.counter = (uint32_t *)c->bws;
    for (int k = 0; k < n; ++k) {
        const stereo_job &j = jobs[order[k]];
        frame_layout(c->p, j.W, j.H, j.Dmax, (char *)c->bws + offs[k], &fw[k]);
        b.job[k] = frame_args(c, fw[k]);
    }
    cudaStream_t us = stream ? (cudaStream_t)stream : c->stream;
    cudaStream_t s = c->stream;
    cudaError_t e;
    if (us != s) {
        if ((e = cudaEventRecord(c->ev_in, us)) != cudaSuccess || (e = cudaStreamWaitEvent(s, c->ev_in, 0)) != cudaSuccess)
            return cuda_fail(c, e, "stream ordering");
    }

    // tile shape: fixed, remembered for this batch signature, or tuned now
    int tile = c->tile;
    int launches = 0;
    if (tile >= 0) {
        for (int k = 0; k < n; ++k)
            if (!costagg_fits(b.job[k], tile)) return fail(c, STEREO_EINVAL, "tile %d does not fit job %d", tile, k);
    } else {
        const std::string sig = batch_signature(c, fw);
        auto it = c->tune.find(sig);
        if (it != c->tune.end()) {
            tile = it->second;
        } else {
            // the autotuner: run the preparation once, then time each tile
            // shape that fits every job (one warm-up and two timed launches)
            for (int k = 0; k < n; ++k)
                if ((e = batch_prep(c, jobs[order[k]], fw[k], s, launches)) != cudaSuccess)
                    return cuda_fail(c, e, "kernel launch");
            float best = 0.f;
            for (int t = 0; t < kNumTiles; ++t) {
                c->last_batch_tune_ms[t] = -1.f;
                bool ok = true;
                for (int k = 0; k < n && ok; ++k) ok = costagg_fits(b.job[k], t);
                if (!ok) continue;
                float tmin = 0.f;
                for (int rep = 0; rep < 3; ++rep) {
                    BatchArgs bt = b;
                    if ((e = cudaEventRecord(c->ev_t0, s)) != cudaSuccess ||
                        (e = launch_costagg_batch(bt, t, c->num_sms, s)) != cudaSuccess ||
                        (e = cudaEventRecord(c->ev_t1, s)) != cudaSuccess ||
                        (e = cudaEventSynchronize(c->ev_t1)) != cudaSuccess)
                        return cuda_fail(c, e, "autotune");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, c->ev_t0, c->ev_t1);
                    if (rep == 1 || (rep > 1 && ms < tmin)) tmin = ms;
                }
                c->last_batch_tune_ms[t] = tmin;
                if (tile < 0 || tmin < best) {
                    best = tmin;
                    tile = t;
                }
            }
            if (tile < 0) return fail(c, STEREO_EINVAL, "no tile shape fits every job of the batch");
            c->tune[sig] = tile;
        }
    }

    // capture the batch as one graph, then update the last graph in place
    launches = 0;
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(c, e, "stream capture");
    for (int k = 0; k < n && e == cudaSuccess; ++k) e = batch_prep(c, jobs[order[k]], fw[k], s, launches);
    if (e == cudaSuccess) {
        e = launch_costagg_batch(b, tile, c->num_sms, s);
        launches++;
    }
    for (int k = 0; k < n && e == cudaSuccess; ++k) e = batch_post(c, jobs[order[k]], fw[k], s, launches);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return cuda_fail(c, e != cudaSuccess ? e : e2, "batch capture");
    }
    // batches of one size share the graph topology, so the last graph of that
    // size is updated in place; a new size or tile shape instantiates anew
    cudaGraphExec_t &exec = c->bexec[n];
    if (exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
    }
    if (!exec && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        exec = nullptr;
        return cuda_fail(c, e, "graph instantiate");
    }
    cudaGraphDestroy(graph);
    if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
    if (us != s) {
        if ((e = cudaEventRecord(c->ev_out, s)) != cudaSuccess || (e = cudaStreamWaitEvent(us, c->ev_out, 0)) != cudaSuccess)
            return cuda_fail(c, e, "stream ordering");
    }
    c->launches = launches;
    c->last_batch_tile = tile;
    return STEREO_OK;
}

size_t stereo_job_bytes(const stereo_params *p, int W, int H, int Dmax)
{
    stereo_params q;
    if (p) q = *p; else stereo_default_params(&q);
    if (check_params(nullptr, q) != STEREO_OK) return 0;
    const int D = q.downscale ? (Dmax + 1) / 2 : Dmax;
    if (W < 1 || H < 1 || W > 8192 || H > 8192 || (q.downscale && (W < 2 || H < 2)) || Dmax < 1 || D > 256 ||
        (q.downscale ? W / 2 : W) > 4096)
        return 0;
    // the frame's layout plus one 256-byte share of the batch's tile counter
    return frame_layout(q, W, H, Dmax, nullptr, nullptr) + 256;
}

int stereo_batch_tile(const stereo_ctx *c, float *tune_ms, int n)
{
    if (!c) return STEREO_EINVAL;
    if (tune_ms)
        for (int i = 0; i < n && i < kNumTiles; ++i) tune_ms[i] = c->last_batch_tune_ms[i];
    return c->last_batch_tile;
}

int stereo_tune_save(stereo_ctx *c, const char *path)
{
    if (!c || !path) return STEREO_EINVAL;
    FILE *f = fopen(path, "w");
    if (!f) return fail(c, STEREO_EINVAL, "cannot write %s", path);
    for (const auto &kv : c->tune) fprintf(f, "%s\t%d\n", kv.first.c_str(), kv.second);
    fclose(f);
    return (int)c->tune.size();
}

int stereo_tune_load(stereo_ctx *c, const char *path)
{
    if (!c || !path) return STEREO_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f) return fail(c, STEREO_EINVAL, "cannot read %s", path);
    char line[1024];
    int n = 0;
    while (fgets(line, sizeof line, f)) {
        char *tab = strrchr(line, '\t');
        if (!tab) continue;
        *tab = '\0';
        const int t = atoi(tab + 1);
        if (t < 0 || t >= kNumTiles) continue;
        c->tune[line] = t;
        ++n;
    }
    fclose(f);
    return n;
}

}  // extern "C"

// ---------------------------------------------------------------- differentiable form

namespace {

int diff_common(stereo_ctx *c, int B, int W, int H, int D, const float *l, const float *r, const uint8_t *lu,
                const uint8_t *ru, const float *theta, float tau, DiffArgs &a)
{
    if (!l || !r || !lu || !ru || !theta) return fail(c, STEREO_EINVAL, "NULL input");
    if (B < 1 || B > 64 || W < 1 || H < 1 || W > 4096 || H > 8192 || D < 1 || D > 256 || !(tau > 0.f))
        return fail(c, STEREO_EINVAL, "bad B, W, H, D or tau");
    const size_t need = diff_workspace_bytes(W, H, c->p.wy, B, D);
    if (need > c->dws_size) {
        if (c->mem_cap && need + c->ws_size + c->bws_size > c->mem_cap)
            return fail(c, STEREO_ENOMEM, "differentiable workspace of %zu bytes exceeds the cap", need);
        if (c->dws) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->dws);
            c->dws = nullptr;
            c->dws_size = 0;
        }
        if (cudaMalloc(&c->dws, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, STEREO_ENOMEM, "cudaMalloc(%zu) failed", need);
        }
        c->dws_size = need;
    }
    a = DiffArgs{};
    a.B = B;
    a.W = W;
    a.H = H;
    a.D = D;
    a.left = l;
    a.right = r;
    a.left_u8 = lu;
    a.right_u8 = ru;
    a.theta = theta;
    a.tau = tau;
    a.ws = c->dws;
    a.err = c->d_err;
    a.wx = c->p.wx;
    a.wy = c->p.wy;
    a.tc = c->p.tc;
    return STEREO_OK;
}

// The differentiable form's ~70 launches per frame, captured on the
// context's stream as one graph (ordered with the caller's stream through
// events) and replayed; the graph of the last call of the same direction is
// updated in place, and instantiated anew when the shapes change.
cudaError_t diff_graph_run(stereo_ctx *c, const DiffArgs &a, cudaStream_t us)
{
    cudaStream_t s = c->stream;
    cudaError_t e;
    if ((e = diff_setup()) != cudaSuccess) return e;
    if (us != s) {
        if ((e = cudaEventRecord(c->ev_in, us)) != cudaSuccess || (e = cudaStreamWaitEvent(s, c->ev_in, 0)) != cudaSuccess)
            return e;
    }
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    e = diff_run(a, s);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return e != cudaSuccess ? e : e2;
    }
    cudaGraphExec_t &exec = c->dexec[a.backward ? 1 : 0];
    if (exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
    }
    if (!exec && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        exec = nullptr;
        return e;
    }
    cudaGraphDestroy(graph);
    if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return e;
    if (us != s) {
        if ((e = cudaEventRecord(c->ev_out, s)) != cudaSuccess || (e = cudaStreamWaitEvent(us, c->ev_out, 0)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int stereo_diff_forward(stereo_ctx *c, int B, int W, int H, int D, const float *left, const float *right,
                        const uint8_t *left_u8, const uint8_t *right_u8, const float *theta, float tau,
                        float *dhat, float *stats, void *stream)
{
    if (!c) return STEREO_EINVAL;
    c->err.clear();
    if (!dhat || !stats) return fail(c, STEREO_EINVAL, "NULL output");
    DeviceGuard g(c->device);
    DiffArgs a;
    int rc = diff_common(c, B, W, H, D, left, right, left_u8, right_u8, theta, tau, a);
    if (rc != STEREO_OK) return rc;
    a.dhat = dhat;
    a.stats = stats;
    a.backward = 0;
    cudaError_t e = diff_graph_run(c, a, stream ? (cudaStream_t)stream : c->stream);
    return e == cudaSuccess ? STEREO_OK : cuda_fail(c, e, "kernel launch");
}

int stereo_diff_backward(stereo_ctx *c, int B, int W, int H, int D, const float *left, const float *right,
                         const uint8_t *left_u8, const uint8_t *right_u8, const float *theta, float tau,
                         const float *dhat, const float *stats, const float *grad_dhat, float *grad_left,
                         float *grad_right, float *grad_theta, void *stream)
{
    if (!c) return STEREO_EINVAL;
    c->err.clear();
    if (!dhat || !stats || !grad_dhat || !grad_left || !grad_right || !grad_theta)
        return fail(c, STEREO_EINVAL, "NULL argument");
    DeviceGuard g(c->device);
    DiffArgs a;
    int rc = diff_common(c, B, W, H, D, left, right, left_u8, right_u8, theta, tau, a);
    if (rc != STEREO_OK) return rc;
    a.dhat = const_cast<float *>(dhat);
    a.stats = const_cast<float *>(stats);
    a.grad_dhat = grad_dhat;
    a.grad_left = grad_left;
    a.grad_right = grad_right;
    a.grad_theta = grad_theta;
    a.backward = 1;
    cudaError_t e = diff_graph_run(c, a, stream ? (cudaStream_t)stream : c->stream);
    return e == cudaSuccess ? STEREO_OK : cuda_fail(c, e, "kernel launch");
}

}  // extern "C"
