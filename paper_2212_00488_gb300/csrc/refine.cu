// Post-processing kernels: GCP cross-check (Eq. 10, Step 6), 3x3 median of
// D^L and bilateral-estimation fill (Eq. 11, Step 7) in one row-resident
// kernel, and the 2x scale-up (Step 8).
#include "internal.cuh"

namespace stereo {
namespace {

constexpr int kRefNT = 256;
constexpr int kMaxRefineX = 4096;   // processed width limit of the row kernel
constexpr int kRefLoads = 4;        // rows up to kRefNT * kRefLoads wide load in one round

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
    if (X <= kRefNT * kRefLoads) {
        // every load of the thread in flight at once
        uint32_t ku[kRefLoads], kc[kRefLoads], kd[kRefLoads], kr[kRefLoads], gv[kRefLoads];
#pragma unroll
        for (int k = 0; k < kRefLoads; ++k) {
            const int x = threadIdx.x + k * kRefNT;
            if (x < X) {
                ku[k] = __ldg(key_l + (size_t)yu * X + x);
                kc[k] = __ldg(key_l + r + x);
                kd[k] = __ldg(key_l + (size_t)yd * X + x);
                kr[k] = __ldg(key_r + r + x);
                gv[k] = __ldg(grey + r + x);
            }
        }
#pragma unroll
        for (int k = 0; k < kRefLoads; ++k) {
            const int x = threadIdx.x + k * kRefNT;
            if (x < X) {
                dlu[x] = (uint8_t)(ku[k] & 0xFF);
                dlc[x] = (uint8_t)(kc[k] & 0xFF);
                dld[x] = (uint8_t)(kd[k] & 0xFF);
                drc[x] = (uint8_t)(kr[k] & 0xFF);
                gr[x] = (uint8_t)gv[k];
            }
        }
    } else {
        for (int x = threadIdx.x; x < X; x += kRefNT) {
            dlu[x] = (uint8_t)(__ldg(key_l + (size_t)yu * X + x) & 0xFF);
            dlc[x] = (uint8_t)(__ldg(key_l + r + x) & 0xFF);
            dld[x] = (uint8_t)(__ldg(key_l + (size_t)yd * X + x) & 0xFF);
            drc[x] = (uint8_t)(__ldg(key_r + r + x) & 0xFF);
            gr[x] = __ldg(grey + r + x);
        }
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

// Step 8: bilateral estimation along x, linear along y; full-resolution
// disparity units (x2). Even output columns 2x take 2 D(x); odd columns
// 2x + 1 between two low-res pixels take D(x) + D(x+1) when those differ by
// at most T, else twice the side whose low-res brightness is strictly closer
// to the full-res pixel's (else the right side). Output rows 2y take low-res
// row y, rows 2y + 1 the mean of rows y and y + 1 (row y at the last row).
// One thread makes the 2x4 outputs (2x..2x+1, 4y'..4y'+3) of low-res column
// x and rows 2y', 2y'+1: it loads everything the three row passes (rows 2y',
// 2y'+1, 2y'+2) may need, brightness included, in one round, so each output
// waits for one memory latency.
template <bool kPairs>
__global__ void upscale_kernel(const float *__restrict__ dp, const uint8_t *__restrict__ gs,
                               const uint8_t *__restrict__ gf, int X, int Y, int W, int H, int T,
                               float *__restrict__ out)
{
    pdl_trigger();
    pdl_wait();                                   // the filled map of the refine kernel
    const int bx = blockIdx.x * blockDim.x + threadIdx.x;
    const int by = 2 * blockIdx.y;                // low-res rows by, by + 1
    const int xo = 2 * bx;
    if (xo >= W || 2 * by >= H) return;
    const bool odd = xo + 1 < W;
    const bool pair = odd && bx + 1 < X;          // odd column between two low-res pixels
    const int xc = min(bx, X - 1);
    float a[3], b[3];
    int gfull[3], ga[3], gb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int yr = min(by + k, Y - 1);
        const float *row = dp + (size_t)yr * X;
        a[k] = __ldg(row + xc);
        b[k] = a[k];
        gfull[k] = ga[k] = gb[k] = 0;
        if (pair) {
            b[k] = __ldg(row + bx + 1);
            gfull[k] = __ldg(gf + (size_t)(2 * yr) * W + xo + 1);
            ga[k] = __ldg(gs + (size_t)yr * X + bx);
            gb[k] = __ldg(gs + (size_t)yr * X + bx + 1);
        }
    }
    // row passes of low-res rows by, by + 1, by + 2 (clamped to the image)
    float e[3], o[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e[k] = __fmul_rn(2.0f, a[k]);
        if (!pair)
            o[k] = e[k];
        else if (fabsf(__fsub_rn(a[k], b[k])) <= (float)T)
            o[k] = __fadd_rn(a[k], b[k]);
        else
            o[k] = __fmul_rn(2.0f, abs(ga[k] - gfull[k]) < abs(gb[k] - gfull[k]) ? a[k] : b[k]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int yo = 2 * (by + k);
        if (yo >= H) break;
        const float e0 = e[k], o0 = o[k];
        float e1 = e0, o1 = o0;
        if (by + k + 1 < Y) {
            e1 = __fmul_rn(0.5f, __fadd_rn(e0, e[k + 1]));
            o1 = __fmul_rn(0.5f, __fadd_rn(o0, o[k + 1]));
        }
        float *r0 = out + (size_t)yo * W + xo;
        if (kPairs) {                               // W even: 8-byte aligned pairs
            *reinterpret_cast<float2 *>(r0) = make_float2(e0, o0);
            if (yo + 1 < H) *reinterpret_cast<float2 *>(r0 + W) = make_float2(e1, o1);
        } else {
            r0[0] = e0;
            if (odd) r0[1] = o0;
            if (yo + 1 < H) {
                r0[W] = e1;
                if (odd) r0[W + 1] = o1;
            }
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
    dim3 grid(((W + 1) / 2 + 127) / 128, ((H + 1) / 2 + 1) / 2);
    const bool pairs = W % 2 == 0 && (reinterpret_cast<uintptr_t>(out) & 7) == 0;
    if (pairs)
        return launch_dependent(upscale_kernel<true>, grid, dim3(128), 0, s, dplus, grey_low, grey_full, X, Y, W, H,
                                T, out);
    return launch_dependent(upscale_kernel<false>, grid, dim3(128), 0, s, dplus, grey_low, grey_full, X, Y, W, H, T,
                            out);
}

}  // namespace stereo
