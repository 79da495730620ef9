// C ABI of the library (include/stereo.h): context, workspace, argument
// checks and the order of the pipeline's kernels (Sec. III steps 1-8).
#include "../../include/stereo.h"
#include "internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

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
    bool prof_events = false;
    ProfSlot prof_ring[kProfRing];
    int prof_next = 0;
    double prof_acc[STEREO_NUM_STAGES] = {};
    int prof_n = 0;
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
    for (int i = 0; i < 2; ++i) c->armc[i] = (uint32_t *)take((size_t)X * (Y + c->p.wy) * 4);
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
        cudaError_t e = launch_grey(c->in_l, c->in_r, c->gf[0], c->gf[1], c->W, c->H, s);
        c->launches++;
        if (e != cudaSuccess || !ds) return e;
        c->launches++;
        return launch_downscale(c->gf[0], c->gf[1], c->gs[0], c->gs[1], c->W, c->H, s);
    }
    case STEREO_STAGE_SUPPORT:
        c->launches += 2;
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
        return launch_refine(c->key[0], c->key[1], c->gs[0], c->X, c->Y, c->p.t_fill, c->out_dl, c->out_dr,
                             c->out_gcp, c->dm, c->dplus, s);
    case STEREO_STAGE_UPSCALE:
        if (!ds) return cudaSuccess;
        c->launches++;
        return launch_upscale(c->dplus, c->gs[0], c->gf[0], c->X, c->Y, c->W, c->H, c->p.t_fill, c->out_disp, s);
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
    if (c->prof) {
        sl = &c->prof_ring[c->prof_next];
        c->prof_next = (c->prof_next + 1) % stereo_ctx::kProfRing;
        cudaError_t e = harvest(c, *sl);
        if (e != cudaSuccess) return cuda_fail(c, e, "profiling events");
    }
    for (int st = 0; st < STEREO_NUM_STAGES; ++st) {
        if (sl) cudaEventRecord(sl->ev[st], s);
        cudaError_t e = run_stage(c, st, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
        if (sl) sl->ran[st] = c->p.downscale || st != STEREO_STAGE_UPSCALE;
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

int stereo_compute_host(stereo_ctx *c, const uint8_t *left_rgb, const uint8_t *right_rgb, int W, int H,
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
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    if (*c->h_err) return fail(c, STEREO_ETIMEOUT, "a bounded wait in the fused kernel gave up");
    return STEREO_OK;
}

int stereo_sync(stereo_ctx *c)
{
    if (!c) return STEREO_EINVAL;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    if ((e = cudaMemcpy(c->h_err, c->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, e, "device-to-host copy");
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
    if (!c) return STEREO_EINVAL;
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
    c->prof = on != 0;
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
    return costagg_pick(a, c->num_sms);
}

}  // extern "C"
