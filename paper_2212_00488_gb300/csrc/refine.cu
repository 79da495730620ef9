// Post-processing kernels: GCP cross-check (Eq. 10, Step 6), 3x3 median of
// D^L, bilateral-estimation fill (Eq. 11, Step 7) and the 2x scale-up
// (Step 8). On the downscaling path one kernel does all four, three low-res
// rows per CTA with the filled rows kept in shared memory; without
// downscaling the row kernel ends at the fill.
#include "internal.cuh"

namespace stereo {
namespace {

constexpr int kRefNT = 256;
constexpr int kMaxRefineX = 4096;   // processed width limit of both refine kernels
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

// Step 7 at a pixel x that is not a GCP, from the nearest GCPs li < x (hl:
// there is one) and ri > x (hr) of its row, the row's medians dm and
// brightness gr.
__device__ __forceinline__ float fill_value(int x, int li, int ri, bool hl, bool hr, const uint8_t *dm,
                                            const uint8_t *gr, int T, int fill_mode)
{
    if (hl && hr) {
        const int i = x - li, j = ri - x;
        const int a = dm[li], b = dm[ri];
        if (fill_mode == 1) return (float)(i < j ? a : b);      // the closer GCP (Fig. 5a)
        if (fill_mode == 2) return (float)min(a, b);            // the smaller disparity (Fig. 5b)
        // linear fill between the two GCPs (Step 7); exact numerator
        if (abs(a - b) <= T) return __fdiv_rn(__int2float_rn(a * j + b * i), __int2float_rn(i + j));
        const int ga = abs((int)gr[li] - (int)gr[x]);
        const int gb = abs((int)gr[ri] - (int)gr[x]);
        return (float)(ga < gb ? a : b);
    }
    if (hl) return (float)dm[li];
    if (hr) return (float)dm[ri];
    return 0.0f;
}

// Step 8 along x, full-resolution units: the odd column 2x + 1 between the
// low-res pixels x (value a, brightness ga) and x + 1 (b, gb) takes a + b
// when they differ by at most T, else twice the side whose low-res
// brightness is strictly closer to the full-res pixel's (gfull), else b.
__device__ __forceinline__ float odd_value(float a, float b, int ga, int gb, int gfull, int T)
{
    if (fabsf(__fsub_rn(a, b)) <= (float)T) return __fadd_rn(a, b);
    return __fmul_rn(2.0f, abs(ga - gfull) < abs(gb - gfull) ? a : b);
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
        const int li = lidx[x], ri = ridx[x];
        const float v = gcp[x] ? (float)dm[x] : fill_value(x, li, ri, li >= 0, ri != 0x7fffffff, dm, gr, T, fill_mode);
        dplus[r + x] = v;
    }
}

// Steps 6-8 in one kernel (the downscaling path). CTA k takes low-res rows
// by = 2k and by + 1 (those below Y) and full-res rows 2 by .. 2 by + 3.
// It cross-checks, takes the medians of and fills low-res rows
// r_j = min(rb + j, Y - 1), j = 0, 1, 2 (rb = min(by, Y - 1)); row r_2 only
// gives the vertical mean of full-res row 2 by + 3 and is filled again by
// the next CTA. The filled rows stay in shared memory for Step 8:
//  * along x: even full-res columns 2x take 2 D(x), odd ones odd_value();
//  * along y: full-res row 2y takes low-res row y, row 2y + 1 the mean of
//    rows y and y + 1 (row y at the last row).
// Every row the CTA reads is requested in one round of loads; the nearest
// GCPs of the three rows come from one block scan over their concatenation.
// The maps, medians and filled rows of low-res rows by and by + 1 are
// written for the debug and map outputs.
constexpr int kRUNT = 256;                 // threads of a CTA
constexpr int kRULoad = 3;                 // columns per thread in one round of loads

template <bool kPairs>
__global__ void __launch_bounds__(kRUNT) refine_up_kernel(
    const uint32_t *__restrict__ key_l, const uint32_t *__restrict__ key_r, const uint8_t *__restrict__ gs,
    const uint8_t *__restrict__ gf, int X, int Y, int W, int H, int T, int fill_mode, uint8_t *dl_out,
    uint8_t *dr_out, uint8_t *gcp_out, uint8_t *dm_out, float *dplus_out, float *__restrict__ out)
{
    extern __shared__ __align__(16) uint8_t sm[];
    pdl_trigger();
    pdl_wait();                                        // the keys of the fused kernel
    const int t = threadIdx.x;
    const int by = 2 * blockIdx.x;
    const int rb = min(by, Y - 1);
    int *scan_sh = reinterpret_cast<int *>(sm);                        // 32 ints
    float *dp = reinterpret_cast<float *>(sm) + 32;                    // [3][X] filled rows
    int16_t *lidx = reinterpret_cast<int16_t *>(dp + 3 * X);          // [3][X] nearest GCP before, -1 if none
    uint8_t *dl5 = reinterpret_cast<uint8_t *>(lidx + 3 * X);         // [5][X] D^L rows clamp(rb - 1 + i)
    uint8_t *dr3 = dl5 + 5 * X, *gr3 = dr3 + 3 * X, *gcp3 = gr3 + 3 * X, *dm3 = gcp3 + 3 * X;
    uint8_t *gfo3 = dm3 + 3 * X;                                      // [3][X] full-res grey at (2 r_j, 2x + 1)

    for (int xb = 0; xb < X; xb += kRULoad * kRUNT) {
        uint32_t v[14][kRULoad];
#pragma unroll
        for (int c = 0; c < kRULoad; ++c) {
            const int x = xb + t + c * kRUNT;
            if (x < X) {
#pragma unroll
                for (int i = 0; i < 5; ++i) v[i][c] = __ldg(key_l + (size_t)min(max(rb - 1 + i, 0), Y - 1) * X + x);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int r = min(rb + j, Y - 1);
                    v[5 + j][c] = __ldg(key_r + (size_t)r * X + x);
                    v[8 + j][c] = __ldg(gs + (size_t)r * X + x);
                    v[11 + j][c] = __ldg(gf + (size_t)(2 * r) * W + 2 * x + 1);   // 2x + 1 < 2X <= W
                }
            }
        }
#pragma unroll
        for (int c = 0; c < kRULoad; ++c) {
            const int x = xb + t + c * kRUNT;
            if (x < X) {
#pragma unroll
                for (int i = 0; i < 5; ++i) dl5[i * X + x] = (uint8_t)(v[i][c] & 0xFF);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    dr3[j * X + x] = (uint8_t)(v[5 + j][c] & 0xFF);
                    gr3[j * X + x] = (uint8_t)v[8 + j][c];
                    gfo3[j * X + x] = (uint8_t)v[11 + j][c];
                }
            }
        }
    }
    __syncthreads();

    // Eq. 10 and the 3x3 median of D^L for the three rows
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int cj = min(rb + j, Y - 1) - rb + 1;   // row r_j of D^L is dl5 row cj; its neighbours cj -+ 1
        const uint8_t *du = dl5 + (cj - 1) * X, *dc = dl5 + cj * X, *dd = dl5 + (cj + 1) * X;
        const uint8_t *drc = dr3 + j * X;
        const bool emit = j < 2 && by + j < Y;
        const size_t ro = (size_t)(by + j) * X;
        for (int x = t; x < X; x += kRUNT) {
            const int k = dc[x];
            const uint8_t isg = (x - k >= 0 && drc[x - k] == k) ? 1 : 0;
            const int xm = max(x - 1, 0), xp = min(x + 1, X - 1);
            const int m = median9(du[xm], du[x], du[xp], dc[xm], dc[x], dc[xp], dd[xm], dd[x], dd[xp]);
            gcp3[j * X + x] = isg;
            dm3[j * X + x] = (uint8_t)m;
            if (emit) {
                if (dl_out) dl_out[ro + x] = (uint8_t)k;
                if (dr_out) dr_out[ro + x] = drc[x];
                if (gcp_out) gcp_out[ro + x] = isg;
                if (dm_out) dm_out[ro + x] = (uint8_t)m;
            }
        }
    }
    __syncthreads();

    // Step 7 over the three rows as one sequence p = j X + x: the nearest GCP
    // before p in the sequence lies in p's row iff it is >= j X, the nearest
    // after p iff it is < (j + 1) X. Thread t owns the chunk [t ch, t ch + ch).
    const int np = 3 * X, ch = (np + kRUNT - 1) / kRUNT;
    const int c0 = min(np, t * ch), c1 = min(np, c0 + ch);
    int last = -1, first = 0x7fffffff;
    for (int q = c0; q < c1; ++q)
        if (gcp3[q]) {
            last = q;
            if (first == 0x7fffffff) first = q;
        }
    int cur = scan_max_excl(last, scan_sh);
    for (int q = c0; q < c1; ++q) {
        lidx[q] = (int16_t)cur;
        if (gcp3[q]) cur = q;
    }
    int cr = scan_min_excl_rev(first, scan_sh);
    int j = (c1 - 1) / X, jx = j * X;          // row of q and its first index
    for (int q = c1 - 1; q >= c0; --q) {
        if (q < jx) {
            --j;
            jx -= X;
        }
        const int li = lidx[q], x = q - jx;
        dp[q] = gcp3[q] ? (float)dm3[q]
                        : fill_value(x, li - jx, cr - jx, li >= jx, cr < jx + X, dm3 + jx, gr3 + jx, T, fill_mode);
        if (gcp3[q]) cr = q;
    }
    __syncthreads();

#pragma unroll
    for (int j = 0; j < 2; ++j)
        if (dplus_out && by + j < Y)
            for (int x = t; x < X; x += kRUNT) dplus_out[(size_t)(by + j) * X + x] = dp[j * X + x];
    // Step 8: low-res column bx makes full-res columns 2 bx, 2 bx + 1 of rows 2 by .. 2 by + 3
    const int nbx = (W + 1) / 2;
    for (int bx = t; bx < nbx; bx += kRUNT) {
        const int xo = 2 * bx;
        const bool odd = xo + 1 < W;
        const bool pair = odd && bx + 1 < X;          // odd column between two low-res pixels
        const int xc = min(bx, X - 1);
        float e[3], o[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float a = dp[k * X + xc];
            e[k] = __fmul_rn(2.0f, a);
            o[k] = pair ? odd_value(a, dp[k * X + bx + 1], gr3[k * X + bx], gr3[k * X + bx + 1], gfo3[k * X + bx], T)
                        : e[k];
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
}

// scan scratch, dp [3][X] float, lidx [3][X] int16, D^L [5][X] and five [3][X]
// byte planes
size_t refine_up_smem(int X) { return 32 * sizeof(int) + (size_t)X * (3 * 4 + 3 * 2 + 5 + 5 * 3); }

size_t refine_smem(int X) { return (size_t)X * (2 * sizeof(int) + 7) + 32 * sizeof(int); }

}  // namespace

cudaError_t refine_setup()
{
    cudaError_t e = cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)refine_smem(kMaxRefineX));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(refine_up_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)refine_up_smem(kMaxRefineX));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(refine_up_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)refine_up_smem(kMaxRefineX));
    return e;
}

cudaError_t launch_refine(const uint32_t *key_l, const uint32_t *key_r, const uint8_t *grey_l,
                          int X, int Y, int T, int fill_mode, uint8_t *dl, uint8_t *dr, uint8_t *gcp,
                          uint8_t *dm, float *dplus, cudaStream_t s)
{
    if (X > kMaxRefineX || fill_mode < 0 || fill_mode > 2) return cudaErrorInvalidValue;
    return launch_dependent(refine_kernel, dim3(Y), dim3(kRefNT), refine_smem(X), s, key_l, key_r, grey_l, X, Y, T,
                            fill_mode, dl, dr, gcp, dm, dplus);
}

cudaError_t launch_refine_up(const uint32_t *key_l, const uint32_t *key_r, const uint8_t *grey_low,
                             const uint8_t *grey_full, int X, int Y, int W, int H, int T, int fill_mode, uint8_t *dl,
                             uint8_t *dr, uint8_t *gcp, uint8_t *dm, float *dplus, float *out, cudaStream_t s)
{
    if (X < 1 || Y < 1 || X > kMaxRefineX || 2 * X > W || 2 * Y > H || fill_mode < 0 || fill_mode > 2)
        return cudaErrorInvalidValue;
    const dim3 grid(((H + 1) / 2 + 1) / 2);
    const size_t smem = refine_up_smem(X);
    if (W % 2 == 0 && (reinterpret_cast<uintptr_t>(out) & 7) == 0)
        return launch_dependent(refine_up_kernel<true>, grid, dim3(kRUNT), smem, s, key_l, key_r, grey_low, grey_full,
                                X, Y, W, H, T, fill_mode, dl, dr, gcp, dm, dplus, out);
    return launch_dependent(refine_up_kernel<false>, grid, dim3(kRUNT), smem, s, key_l, key_r, grey_low, grey_full, X,
                            Y, W, H, T, fill_mode, dl, dr, gcp, dm, dplus, out);
}

}  // namespace stereo
