// Post-processing kernels: GCP cross-check (Eq. 10, Step 6), 3x3 median of
// D^L and bilateral-estimation fill (Eq. 11, Step 7) in one row-resident
// kernel, and the 2x scale-up (Step 8).
#include "internal.cuh"

namespace stereo {
namespace {

constexpr int kRefNT = 256;
constexpr int kMaxRefineX = 4096;   // processed width limit of the row kernel

__device__ __forceinline__ int med3(int a, int b, int c)
{
    return max(min(a, b), min(max(a, b), c));
}

// Median of nine values: the classic exchange network on three sorted rows.
__device__ __forceinline__ int median9(int v0, int v1, int v2, int v3, int v4, int v5, int v6, int v7, int v8)
{
    // sort each triple
    int a0 = min(min(v0, v1), v2), a2 = max(max(v0, v1), v2), a1 = v0 + v1 + v2 - a0 - a2;
    int b0 = min(min(v3, v4), v5), b2 = max(max(v3, v4), v5), b1 = v3 + v4 + v5 - b0 - b2;
    int c0 = min(min(v6, v7), v8), c2 = max(max(v6, v7), v8), c1 = v6 + v7 + v8 - c0 - c2;
    // the median is the median of (max of mins, median of medians, min of maxes)
    int lo = max(max(a0, b0), c0);
    int mi = med3(a1, b1, c1);
    int hi = min(min(a2, b2), c2);
    return med3(lo, mi, hi);
}

// Block-wide exclusive max scan over threads (value of threads < tid), and
// exclusive min scan from the other side (threads > tid).
__device__ int scan_max_excl(int v, int *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl = max(incl, t);
    }
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    int carry = -1;
    for (int w = 0; w < warp; ++w) carry = max(carry, sh[w]);
    int prev = __shfl_up_sync(0xffffffffu, incl, 1);
    int excl = lane ? max(prev, carry) : carry;
    __syncthreads();
    return excl;
}

__device__ int scan_min_excl_rev(int v, int *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_down_sync(0xffffffffu, incl, o);
        if (lane + o < 32) incl = min(incl, t);
    }
    if (lane == 0) sh[warp] = incl;
    __syncthreads();
    int carry = 0x7fffffff;
    for (int w = warp + 1; w < nw; ++w) carry = min(carry, sh[w]);
    int next = __shfl_down_sync(0xffffffffu, incl, 1);
    int excl = lane < 31 ? min(next, carry) : carry;
    __syncthreads();
    return excl;
}

// One CTA per processed row y.
__global__ void __launch_bounds__(kRefNT) refine_kernel(
    const uint32_t *__restrict__ key_l, const uint32_t *__restrict__ key_r,
    const uint8_t *__restrict__ grey, int X, int Y, int T, int fill_mode,
    uint8_t *dl_out, uint8_t *dr_out, uint8_t *gcp_out, uint8_t *dm_out, float *__restrict__ dplus)
{
    extern __shared__ __align__(16) uint8_t sm[];
    pdl_trigger();
    pdl_wait();                                        // the keys of the fused kernel
    int *lidx = reinterpret_cast<int *>(sm);           // nearest GCP strictly left, -1 if none
    int *ridx = lidx + X;                              // nearest GCP strictly right, INT_MAX if none
    int *scan_sh = ridx + X;                           // 32 ints
    uint8_t *dlu = reinterpret_cast<uint8_t *>(scan_sh + 32);
    uint8_t *dlc = dlu + X, *dld = dlc + X, *drc = dld + X, *gcp = drc + X, *dm = gcp + X, *gr = dm + X;

    const int y = blockIdx.x;
    const int yu = max(y - 1, 0), yd = min(y + 1, Y - 1);
    const size_t r = (size_t)y * X;
    for (int x = threadIdx.x; x < X; x += kRefNT) {
        dlu[x] = (uint8_t)(__ldg(key_l + (size_t)yu * X + x) & 0xFF);
        dlc[x] = (uint8_t)(__ldg(key_l + r + x) & 0xFF);
        dld[x] = (uint8_t)(__ldg(key_l + (size_t)yd * X + x) & 0xFF);
        drc[x] = (uint8_t)(__ldg(key_r + r + x) & 0xFF);
        gr[x] = __ldg(grey + r + x);
    }
    __syncthreads();

    for (int x = threadIdx.x; x < X; x += kRefNT) {
        const int k = dlc[x];
        const uint8_t isg = (x - k >= 0 && drc[x - k] == k) ? 1 : 0;   // Eq. 10
        gcp[x] = isg;
        const int xm = max(x - 1, 0), xp = min(x + 1, X - 1);
        const int m = median9(dlu[xm], dlu[x], dlu[xp], dlc[xm], dlc[x], dlc[xp], dld[xm], dld[x], dld[xp]);
        dm[x] = (uint8_t)m;
        if (dl_out) dl_out[r + x] = (uint8_t)k;
        if (dr_out) dr_out[r + x] = drc[x];
        if (gcp_out) gcp_out[r + x] = isg;
        if (dm_out) dm_out[r + x] = (uint8_t)m;
    }
    __syncthreads();

    // Nearest GCPs to the left and right of every pixel of the row: each
    // thread owns a contiguous chunk; a block scan carries the last (first)
    // GCP index across chunks.
    const int chunk = (X + kRefNT - 1) / kRefNT;
    const int c0 = threadIdx.x * chunk, c1 = min(X, c0 + chunk);
    int last = -1, first = 0x7fffffff;
    for (int x = c0; x < c1; ++x)
        if (gcp[x]) { last = x; if (first == 0x7fffffff) first = x; }
    int cur = scan_max_excl(last, scan_sh);
    for (int x = c0; x < c1; ++x) { lidx[x] = cur; if (gcp[x]) cur = x; }
    cur = scan_min_excl_rev(first, scan_sh);
    for (int x = c1 - 1; x >= c0; --x) { ridx[x] = cur; if (gcp[x]) cur = x; }
    __syncthreads();

    for (int x = threadIdx.x; x < X; x += kRefNT) {
        float v;
        if (gcp[x]) {
            v = (float)dm[x];
        } else {
            const int li = lidx[x], ri = ridx[x];
            const bool hl = li >= 0, hr = ri != 0x7fffffff;
            if (hl && hr) {
                const int i = x - li, j = ri - x;
                const int a = dm[li], b = dm[ri];
                if (fill_mode == 1) {
                    v = (float)(i < j ? a : b);           // the closer GCP (Fig. 5a)
                } else if (fill_mode == 2) {
                    v = (float)min(a, b);                 // the smaller disparity (Fig. 5b)
                } else if (abs(a - b) <= T) {
                    // linear fill between the two GCPs (Step 7); exact numerator
                    v = __fdiv_rn(__int2float_rn(a * j + b * i), __int2float_rn(i + j));
                } else {
                    const int ga = abs((int)gr[li] - (int)gr[x]);
                    const int gb = abs((int)gr[ri] - (int)gr[x]);
                    v = (float)(ga < gb ? a : b);
                }
            } else if (hl) {
                v = (float)dm[li];
            } else if (hr) {
                v = (float)dm[ri];
            } else {
                v = 0.0f;
            }
        }
        dplus[r + x] = v;
    }
}

// Step 8 row pass for low-res row y at output column xo (see upscale_kernel).
__device__ __forceinline__ float rowpass(const float *__restrict__ dp, const uint8_t *__restrict__ gs,
                                         const uint8_t *__restrict__ gf, int X, int W, int T, int xo, int y)
{
    const int x = xo >> 1;
    const float *row = dp + (size_t)y * X;
    if ((xo & 1) == 0 || x + 1 >= X) return __fmul_rn(2.0f, __ldg(row + min(x, X - 1)));
    const float a = __ldg(row + x), b = __ldg(row + x + 1);
    if (fabsf(__fsub_rn(a, b)) <= (float)T) return __fadd_rn(a, b);
    const int gfull = __ldg(gf + (size_t)(2 * y) * W + xo);
    const int ga = abs((int)__ldg(gs + (size_t)y * X + x) - gfull);
    const int gb = abs((int)__ldg(gs + (size_t)y * X + x + 1) - gfull);
    return __fmul_rn(2.0f, ga < gb ? a : b);
}

// Step 8: bilateral estimation along x, linear along y; full-resolution
// disparity units (x2). Odd output columns between two low-res pixels whose
// disparities differ by more than T take the side whose low-res brightness is
// strictly closer to the full-res pixel's (else the right side). One thread
// makes the 2x2 outputs (2x..2x+1, 2y..2y+1) of low-res position (x, y), so
// each row pass is computed once.
template <bool kPairs>
__global__ void upscale_kernel(const float *__restrict__ dp, const uint8_t *__restrict__ gs,
                               const uint8_t *__restrict__ gf, int X, int Y, int W, int H, int T,
                               float *__restrict__ out)
{
    pdl_trigger();
    pdl_wait();                                   // the filled map of the refine kernel
    const int bx = blockIdx.x * blockDim.x + threadIdx.x;
    const int by = blockIdx.y;
    const int xo = 2 * bx, yo = 2 * by;
    if (xo >= W || yo >= H) return;
    const int yc = min(by, Y - 1);
    float e0 = rowpass(dp, gs, gf, X, W, T, xo, yc);
    float o0 = xo + 1 < W ? rowpass(dp, gs, gf, X, W, T, xo + 1, yc) : 0.f;
    float e1 = e0, o1 = o0;
    if (by + 1 < Y) {
        const float e2 = rowpass(dp, gs, gf, X, W, T, xo, by + 1);
        const float o2 = xo + 1 < W ? rowpass(dp, gs, gf, X, W, T, xo + 1, by + 1) : 0.f;
        e1 = __fmul_rn(0.5f, __fadd_rn(e0, e2));
        o1 = __fmul_rn(0.5f, __fadd_rn(o0, o2));
    }
    float *r0 = out + (size_t)yo * W + xo;
    if (kPairs) {                                   // W even: 8-byte aligned pairs
        *reinterpret_cast<float2 *>(r0) = make_float2(e0, o0);
        if (yo + 1 < H) *reinterpret_cast<float2 *>(r0 + W) = make_float2(e1, o1);
    } else {
        r0[0] = e0;
        if (xo + 1 < W) r0[1] = o0;
        if (yo + 1 < H) {
            r0[W] = e1;
            if (xo + 1 < W) r0[W + 1] = o1;
        }
    }
}

size_t refine_smem(int X) { return (size_t)X * (2 * sizeof(int) + 7) + 32 * sizeof(int); }

}  // namespace

cudaError_t refine_setup()
{
    return cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)refine_smem(kMaxRefineX));
}

cudaError_t launch_refine(const uint32_t *key_l, const uint32_t *key_r, const uint8_t *grey_l,
                          int X, int Y, int T, int fill_mode, uint8_t *dl, uint8_t *dr, uint8_t *gcp,
                          uint8_t *dm, float *dplus, cudaStream_t s)
{
    if (X > kMaxRefineX || fill_mode < 0 || fill_mode > 2) return cudaErrorInvalidValue;
    return launch_dependent(refine_kernel, dim3(Y), dim3(kRefNT), refine_smem(X), s, key_l, key_r, grey_l, X, Y, T,
                            fill_mode, dl, dr, gcp, dm, dplus);
}

cudaError_t launch_upscale(const float *dplus, const uint8_t *grey_low, const uint8_t *grey_full,
                           int X, int Y, int W, int H, int T, float *out, cudaStream_t s)
{
    dim3 grid(((W + 1) / 2 + 127) / 128, (H + 1) / 2);
    const bool pairs = W % 2 == 0 && (reinterpret_cast<uintptr_t>(out) & 7) == 0;
    if (pairs)
        return launch_dependent(upscale_kernel<true>, grid, dim3(128), 0, s, dplus, grey_low, grey_full, X, Y, W, H,
                                T, out);
    return launch_dependent(upscale_kernel<false>, grid, dim3(128), 0, s, dplus, grey_low, grey_full, X, Y, W, H, T,
                            out);
}

}  // namespace stereo
