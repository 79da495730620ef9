// stereo_compute_noalloc: the whole pipeline without any allocation at call
// time. Every intermediate (grey planes, support words, WTA keys, cost tables,
// the error word of the fused kernel's bounded waits) lives in one fixed
// file-scope device array that every GPU loading this library holds until the
// process exits. The kernels are the same as stereo_compute's.
#include "../../include/stereo.h"
#include "internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

using namespace stereo;

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device. The symbol's name in host code is
// only a host-side stand-in, so the address is fetched with
// cudaGetSymbolAddress once per device, with that device current.
unsigned char *g_scratch_dev[kMaxDevices];
bool g_ready[kMaxDevices];
std::mutex g_setup_mutex;

int say(char *err, size_t len, int code, const char *fmt, ...)
{
    if (err && len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, len, fmt, ap);
        va_end(ap);
    }
    return code;
}

int setup_device(int dev, char *err, size_t len)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_ready[dev]) return STEREO_OK;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return say(err, len, STEREO_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    if ((e = costagg_setup()) != cudaSuccess || (e = refine_setup()) != cudaSuccess)
        return say(err, len, STEREO_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    g_ready[dev] = true;
    return STEREO_OK;
}

size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

extern "C" int stereo_compute_noalloc(const stereo_params *params, const uint8_t *left_rgb,
                                      const uint8_t *right_rgb, int W, int H, int Dmax, float *disp_out,
                                      uint8_t *dl_out, uint8_t *dr_out, uint8_t *gcp_out, void *stream,
                                      char *err, size_t err_len)
{
    if (err && err_len) err[0] = '\0';
    stereo_params p;
    if (params) p = *params; else stereo_default_params(&p);
    if (!left_rgb || !right_rgb || !disp_out)
        return say(err, err_len, STEREO_EINVAL, "left, right and disp_out must not be NULL");
    if (!(p.lambda_ad > 0) || !(p.lambda_mc > 0) || p.tc < 0 || p.tc > 256 || p.wx < 0 || p.wx > kMaxWx ||
        p.wy < 0 || p.wy > kMaxWy || p.t_fill < 0 || p.t_fill > 255 || (p.downscale != 0 && p.downscale != 1) ||
        p.fill_mode < 0 || p.fill_mode > 2 ||
        p.cost_scale < 1 || p.cost_scale > (1 << 20))
        return say(err, err_len, STEREO_EINVAL, "parameter out of range");
    const double pmax = p.cost_scale * ((1.0 - std::exp(-1.0 / p.lambda_ad)) + (1.0 - std::exp(-6.0 / p.lambda_mc))) + 1.0;
    if (pmax > 65535.0 || (double)(2 * p.wx + 1) * (2 * p.wy + 1) * pmax >= 16777216.0)
        return say(err, err_len, STEREO_EINVAL, "cost_scale too large for the arm caps");
    if (W < 1 || H < 1 || W > 8192 || H > 8192 || (p.downscale && (W < 2 || H < 2)))
        return say(err, err_len, STEREO_EINVAL, "bad image size %dx%d", W, H);
    const bool ds = p.downscale != 0;
    const int X = ds ? W / 2 : W, Y = ds ? H / 2 : H, D = ds ? (Dmax + 1) / 2 : Dmax;
    if (Dmax < 1 || D > 256 || X > 4096) return say(err, err_len, STEREO_EINVAL, "bad Dmax or width");

    // layout in the fixed scratch array
    const size_t nf = (size_t)W * H, nl = (size_t)X * Y;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += up256(bytes); return o; };
    const size_t o_lut = take(264 * 4), o_err = take(4);
    size_t o_gf[2], o_gs[2], o_pix[2], o_arm[2], o_armc[2], o_key[2];
    for (int i = 0; i < 2; ++i) o_gf[i] = take(nf);
    for (int i = 0; i < 2; ++i) o_gs[i] = ds ? take(nl) : o_gf[i];
    for (int i = 0; i < 2; ++i) o_pix[i] = take(nl * 4);
    for (int i = 0; i < 2; ++i) o_arm[i] = take(nl * 4);
    for (int i = 0; i < 2; ++i) o_armc[i] = take(armc_words(X, Y, p.wy) * 4);
    for (int i = 0; i < 2; ++i) o_key[i] = take(nl * 4);
    const size_t o_dm = take(nl), o_dplus = take(nl * 4);
    if (off > kScratchBytes)
        return say(err, err_len, STEREO_ENOMEM,
                   "a %dx%d frame needs %zu bytes of scratch, more than the fixed %zu", W, H, off, kScratchBytes);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return say(err, err_len, STEREO_ECUDA, "no current CUDA device");
    int rc = setup_device(dev, err, err_len);
    if (rc != STEREO_OK) return rc;
    unsigned char *base = g_scratch_dev[dev];
    cudaStream_t s = (cudaStream_t)stream;

    // cost tables (Eqs. 4-5), quantised on the host exactly as stereo_create does
    uint32_t lut[264];
    for (int a = 0; a < 256; ++a)
        lut[a] = (uint32_t)std::llround(p.cost_scale * (1.0 - std::exp(-((double)a / 255.0) / p.lambda_ad)));
    for (int h = 0; h <= 6; ++h)
        lut[256 + h] = (uint32_t)std::llround(p.cost_scale * (1.0 - std::exp(-(double)h / p.lambda_mc)));
    lut[263] = lut[262];
    if ((e = cudaMemcpyAsync(base + o_lut, lut, sizeof lut, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return say(err, err_len, STEREO_ECUDA, "table copy: %s", cudaGetErrorString(e));

    auto u8 = [&](size_t o) { return reinterpret_cast<uint8_t *>(base + o); };
    auto u32 = [&](size_t o) { return reinterpret_cast<uint32_t *>(base + o); };
    float *dplus = ds ? reinterpret_cast<float *>(base + o_dplus) : disp_out;

    int launches = 0;
    if ((e = ds ? launch_grey_down(left_rgb, right_rgb, u8(o_gf[0]), u8(o_gf[1]), u8(o_gs[0]), u8(o_gs[1]), W, H,
                                   s, &launches)
                : launch_grey(left_rgb, right_rgb, u8(o_gf[0]), u8(o_gf[1]), W, H, s)) == cudaSuccess &&
        (e = launch_support(u8(o_gs[0]), u8(o_gs[1]), u32(o_pix[0]), u32(o_pix[1]), u32(o_arm[0]), u32(o_arm[1]),
                            u32(o_armc[0]), u32(o_armc[1]), u32(o_key[0]), u32(o_key[1]), u32(o_err), X, Y, p.wx,
                            p.wy, p.tc, s)) == cudaSuccess) {
        CostAggArgs a{};
        a.pix_l = u32(o_pix[0]);
        a.pix_r = u32(o_pix[1]);
        a.arm_l = u32(o_arm[0]);
        a.arm_r = u32(o_arm[1]);
        a.armc_l = u32(o_armc[0]);
        a.armc_r = u32(o_armc[1]);
        a.key_l = u32(o_key[0]);
        a.key_r = u32(o_key[1]);
        a.lut_ad = u32(o_lut);
        a.lut_mc = u32(o_lut) + 256;
        a.err = u32(o_err);
        a.wait_limit = 1u << 20;
        a.X = X;
        a.Y = Y;
        a.D = D;
        a.wx = p.wx;
        a.wy = p.wy;
        a.P = lut[255] + lut[256 + 6];
        a.tile = -1;
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        a.num_sms = nsm;
        if ((e = launch_costagg(a, s)) == cudaSuccess)
            e = ds ? launch_refine_up(u32(o_key[0]), u32(o_key[1]), u8(o_gs[0]), u8(o_gf[0]), X, Y, W, H, p.t_fill,
                                      p.fill_mode, dl_out, dr_out, gcp_out, u8(o_dm), dplus, disp_out, s)
                   : launch_refine(u32(o_key[0]), u32(o_key[1]), u8(o_gs[0]), X, Y, p.t_fill, p.fill_mode, dl_out, dr_out,
                                   gcp_out, u8(o_dm), dplus, s);
    }
    if (e != cudaSuccess) return say(err, err_len, STEREO_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return STEREO_OK;
}
