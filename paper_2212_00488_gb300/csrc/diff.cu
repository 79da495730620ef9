// Differentiable form of the left-base cost and aggregation (FP32): a soft
// argmin over the aggregated cost, and its backward as the adjoint of the
// cross aggregation over the same frozen supports.
//
//   g          = (77 R + 150 G + 29 B) / 256 on [0, 1]       (float grey)
//   census codes and arms: frozen (not differentiated), computed by the
//              integer path from the pair's uint8 images
//   C(x,y,d)   = w_AD (1 - exp(-|gL(x,y) - gR(x-d,y)| / l_AD))
//              + w_MC (1 - exp(-MC / l_MC))                    (Eqs. 3-5)
//              = P(theta) when x < d
//   CA(x,y,d)  = Eqs. 7-8 over the frozen arms, divided by the support size
//   dhat       = sum_d d softmax_d(-CA / tau)
//
// The volume is never stored: forward and backward walk the disparities in
// chunks of kDC, keeping per chunk the x-aggregated slab and, in backward,
// the slab's gradients. Every pair of the batch has its own buffers, and the
// per-chunk kernels take all pairs in one launch (blockIdx.y = pair), so a
// launch is several waves of blocks rather than one and a partial one. Sums
// over arms are direct (at most 2 wx + 1 and 2 wy + 1 terms), which keeps FP32
// aggregates within about 6e-6 of their exact value. The adjoint of each sum
// is a banded difference array walked in a fixed order by one thread, so no
// float atomics are used and results are deterministic.
#include "internal.cuh"

namespace stereo {

constexpr int kDiffNT = 256;   // threads of the per-pixel kernels

namespace {

constexpr int kDC = 8;   // disparities per chunk
// pixel tiles of the kernels that sum along y (blocks of kTileX * kTileY = 256 threads)
constexpr int kTileX = 32, kTileY = 8;
__constant__ float kGreyW[3] = {77.f / 256.f, 150.f / 256.f, 29.f / 256.f};

__global__ void diff_grey_kernel(const float *__restrict__ rgb_l, const float *__restrict__ rgb_r,
                                 float *__restrict__ g_l, float *__restrict__ g_r, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t b = blockIdx.z;                  // pair
    rgb_l += b * n * 3;
    rgb_r += b * n * 3;
    g_l += b * n;
    g_r += b * n;
    const float *rgb = blockIdx.y ? rgb_r : rgb_l;
    float g = __fmul_rn(kGreyW[0], rgb[3 * i]);
    g = __fadd_rn(g, __fmul_rn(kGreyW[1], rgb[3 * i + 1]));
    g = __fadd_rn(g, __fmul_rn(kGreyW[2], rgb[3 * i + 2]));
    (blockIdx.y ? g_r : g_l)[i] = g;
}

// Support size n(x,y) = sum over the vertical span of each row's x window.
__global__ void diff_nsupport_kernel(const uint32_t *__restrict__ arm, int X, int Y, float *__restrict__ ns)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= X * Y) return;
    const size_t b = blockIdx.y;                  // pair
    arm += b * X * Y;
    ns += b * X * Y;
    const int y = i / X, x = i - y * X;
    const uint32_t a = arm[i];
    const int up = (a >> 16) & 0xFF, down = a >> 24;
    int s = 0;
    for (int t = -up; t <= down; ++t) {
        const uint32_t b = arm[(size_t)(y + t) * X + x];
        s += (int)(b & 0xFF) + (int)((b >> 8) & 0xFF) + 1;
    }
    ns[i] = (float)s;
}

struct Theta {
    float wad, wmc, lad, lmc;
};

__device__ __forceinline__ Theta load_theta(const float *t) { return Theta{t[0], t[1], t[2], t[3]}; }

// One block per row y and chunk: the cost rows of all disparities of the
// chunk in shared memory ([dc][X]), then each pixel's own x window summed
// directly, every plane in ascending x.
__global__ void diff_costx_kernel(const float *__restrict__ gL, const float *__restrict__ gR,
                                  const uint32_t *__restrict__ pixL, const uint32_t *__restrict__ pixR,
                                  const uint32_t *__restrict__ arm, const float *__restrict__ theta, int X, int Y,
                                  int D, int d0, int dc, float *__restrict__ cax)
{
    extern __shared__ float crow[];
    const int y = blockIdx.x;
    const size_t b = blockIdx.y, n = (size_t)X * Y;   // pair
    gL += b * n;
    gR += b * n;
    pixL += b * n;
    pixR += b * n;
    arm += b * n;
    cax += b * kDC * n;
    const Theta th = load_theta(theta);
    const float P = th.wad * (1.f - expf(-1.f / th.lad)) + th.wmc * (1.f - expf(-6.f / th.lmc));
    const size_t r = (size_t)y * X;
    const int kn = min(dc, D - d0);
    // the census term takes seven values: one exp per Hamming distance
    __shared__ float mc[8];
    if (threadIdx.x < 7) mc[threadIdx.x] = th.wmc * (1.f - expf(-(float)threadIdx.x / th.lmc));
    const float inv_lad = 1.f / th.lad;
    __syncthreads();
    for (int x = threadIdx.x; x < X; x += blockDim.x) {
        const float gl = gL[r + x];
        const uint32_t pl = pixL[r + x];
        // the chunk's disparities unrolled, so their loads and exps overlap
#pragma unroll
        for (int k = 0; k < kDC; ++k) {
            if (k < kn) {
                const int d = d0 + k;
                float c = P;
                if (x >= d) {
                    const float a = fabsf(gl - gR[r + x - d]);
                    const int h = __popc((pl ^ pixR[r + x - d]) & 0x3F00u);
                    c = th.wad * (1.f - expf(-a * inv_lad)) + mc[h];
                }
                crow[k * X + x] = c;
            }
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < X; x += blockDim.x) {
        const uint32_t am = arm[r + x];
        const int lo = x - (int)(am & 0xFF), hi = x + (int)((am >> 8) & 0xFF);
        float s[kDC];
#pragma unroll
        for (int k = 0; k < kDC; ++k) s[k] = 0.f;
        for (int t = lo; t <= hi; ++t) {
#pragma unroll
            for (int k = 0; k < kDC; ++k)
                if (k < kn) s[k] += crow[k * X + t];
        }
#pragma unroll
        for (int k = 0; k < kDC; ++k)
            if (k < kn) cax[((size_t)k * Y + y) * X + x] = s[k];
    }
}

// Vertical sums of Eq. 8 for the chunk's dc planes at once: one pass over the
// anchor's span [y - up, y + down], each plane summed in ascending y.
__device__ __forceinline__ void vsum_chunk(const float *__restrict__ cax, const uint32_t am, int x, int y, int X,
                                           size_t plane, int dc, float (&out)[kDC])
{
    const int up = (am >> 16) & 0xFF, down = am >> 24;
#pragma unroll
    for (int k = 0; k < kDC; ++k) out[k] = 0.f;
    for (int t = -up; t <= down; ++t) {
        const float *p = cax + (size_t)(y + t) * X + x;
#pragma unroll
        for (int k = 0; k < kDC; ++k)
            if (k < dc) out[k] += p[k * plane];
    }
}

// Forward: aggregated cost along y per pixel and an online softmax over d.
// state = (max z, sum exp(z - max), sum d exp(z - max)) per pixel.
__global__ void diff_vagg_softmax_kernel(const float *__restrict__ cax, const uint32_t *__restrict__ arm,
                                         const float *__restrict__ ns, int X, int Y, int D, int d0, int dc,
                                         float inv_tau, float *__restrict__ state, int first, int last,
                                         float *__restrict__ dhat, float *__restrict__ stats)
{
    // 2-D tiles of kTileX x kTileY pixels: the warps of a block walk the
    // same anchor rows, so their vertical windows meet in L1
    const int x = blockIdx.x * kTileX + (int)(threadIdx.x % kTileX);
    const int y = blockIdx.y * kTileY + (int)(threadIdx.x / kTileX);
    if (x >= X || y >= Y) return;
    const int i = y * X + x;
    const size_t b = blockIdx.z, n = (size_t)X * Y;   // pair
    cax += b * kDC * n;
    arm += b * n;
    ns += b * n;
    state += b * 3 * n;
    dhat += b * n;
    stats += b * 2 * n;
    const uint32_t am = arm[i];
    const float inv_n = 1.f / ns[i];
    float m = first ? -INFINITY : state[3 * i], s = first ? 0.f : state[3 * i + 1],
          sd = first ? 0.f : state[3 * i + 2];
    float ca[kDC];
    vsum_chunk(cax, am, x, y, X, (size_t)X * Y, min(dc, D - d0), ca);
#pragma unroll
    for (int k = 0; k < kDC; ++k) {
        if (k >= dc || d0 + k >= D) break;
        const float z = -(ca[k] * inv_n) * inv_tau;
        const float d = (float)(d0 + k);
        if (z > m) {
            const float f = expf(m - z);
            s = s * f + 1.f;
            sd = sd * f + d;
            m = z;
        } else {
            const float e = expf(z - m);
            s += e;
            sd += d * e;
        }
    }
    if (last) {
        dhat[i] = sd / s;
        stats[2 * i] = m;
        stats[2 * i + 1] = s;
    } else {
        state[3 * i] = m;
        state[3 * i + 1] = s;
        state[3 * i + 2] = sd;
    }
}

// Backward 1: d dhat / d CA = p_d (d - dhat) (-1/tau) / n, times the
// incoming gradient, for the chunk (the aggregated slab is recomputed).
__global__ void diff_gca_kernel(const float *__restrict__ cax, const uint32_t *__restrict__ arm,
                                const float *__restrict__ ns, int X, int Y, int D, int d0, int dc, float inv_tau,
                                const float *__restrict__ dhat, const float *__restrict__ stats,
                                const float *__restrict__ go, float *__restrict__ g0)
{
    // 2-D tiles of kTileX x kTileY pixels: the warps of a block walk the
    // same anchor rows, so their vertical windows meet in L1
    const int x = blockIdx.x * kTileX + (int)(threadIdx.x % kTileX);
    const int y = blockIdx.y * kTileY + (int)(threadIdx.x / kTileX);
    if (x >= X || y >= Y) return;
    const int i = y * X + x;
    const size_t b = blockIdx.z, n = (size_t)X * Y;   // pair
    cax += b * kDC * n;
    arm += b * n;
    ns += b * n;
    dhat += b * n;
    stats += b * 2 * n;
    go += b * n;
    g0 += b * kDC * n;
    const uint32_t am = arm[i];
    const float inv_n = 1.f / ns[i];
    const float m = stats[2 * i], s = stats[2 * i + 1], e = dhat[i], gi = go[i];
    float ca[kDC];
    vsum_chunk(cax, am, x, y, X, (size_t)X * Y, min(dc, D - d0), ca);
#pragma unroll
    for (int k = 0; k < kDC; ++k) {
        if (k >= dc) break;
        float v = 0.f;
        if (d0 + k < D) {
            const float z = -(ca[k] * inv_n) * inv_tau;
            const float p = expf(z - m) / s;
            v = gi * p * ((float)(d0 + k) - e) * (-inv_tau) * inv_n;
        }
        g0[(size_t)k * X * Y + i] = v;
    }
}

// Backward 2: adjoint of the vertical sum. G1(x, y') collects the anchors
// (x, y) whose span [y - up, y + down] contains y'. As a difference array: a
// thread owns one column and one disparity of the chunk over a band of kVB
// rows; every anchor whose span reaches the band adds its value at the band
// row where the span enters and subtracts it one row past where the span
// ends (anchors in ascending y), and a running sum down the band gives G1.
// Each thread works alone in a fixed order: deterministic, no atomics, and
// about 2 (kVB + 2 wy) / kVB operations per output instead of 2 wy + 1.
constexpr int kVB = 32;
static_assert(kDiffNT == 32 * kDC, "a block is 32 columns x the chunk's disparities");
__global__ void __launch_bounds__(kDiffNT) diff_vT_kernel(const float *__restrict__ g0,
                                                          const uint32_t *__restrict__ arm, int X, int Y, int wy,
                                                          int dc, float *__restrict__ g1)
{
    __shared__ float delta[kDiffNT][kVB + 1];     // odd pitch: the lanes of a warp hit distinct banks
    const int xi = threadIdx.x % 32, k = threadIdx.x / 32;   // 32 columns x kDC disparities
    const int x = blockIdx.x * 32 + xi, y0 = blockIdx.y * kVB;
    if (x >= X || k >= dc) return;
    const size_t b = blockIdx.z, n = (size_t)X * Y;   // pair
    arm += b * n;
    const float *gp = g0 + b * kDC * n + (size_t)k * n + x;
    float *out = g1 + b * kDC * n + (size_t)k * n + x;
    float *dl = delta[threadIdx.x];
    const int ye = min(y0 + kVB, Y);              // band rows [y0, ye)
#pragma unroll
    for (int i = 0; i <= kVB; ++i) dl[i] = 0.f;
    const int ya = max(y0 - wy, 0), yb = min(ye - 1 + wy, Y - 1);
#pragma unroll 4
    for (int y = ya; y <= yb; ++y) {
        const uint32_t am = arm[(size_t)y * X + x];
        const float v = gp[(size_t)y * X];           // rows [ya, yb] are in the image: loaded ahead of the test
        const int lo = y - (int)((am >> 16) & 0xFF), hi = y + (int)(am >> 24);
        if (hi >= y0 && lo < ye) {
            dl[max(lo, y0) - y0] += v;
            if (hi + 1 < ye) dl[hi + 1 - y0] -= v;
        }
    }
    float s = 0.f;
    for (int i = 0; i < ye - y0; ++i) {
        s += dl[i];
        out[(size_t)(y0 + i) * X] = s;
    }
}

// Backward 3: adjoint of the horizontal sum. G2(x', y) collects the pixels
// (x, y) whose own window [x - left, x + right] contains x'. A block takes one
// row segment of up to kHSeg columns of one pair: it stages the chunk's
// disparity planes and the arm words of the segment and its wx-column halo in
// shared memory (coalesced loads), then, as in the vertical adjoint, a thread
// owns one disparity and a band of 32 columns: each pixel whose window reaches
// the band adds its value where the window enters and subtracts it one column
// past where it ends (pixels in ascending x), and a running sum gives the
// band. The staged rows skip a word every 32, so the 32 bands of a warp,
// 32 columns apart, read distinct banks. The outputs go back through shared
// memory and leave in coalesced rows.
constexpr int kHSeg = 1024;                       // 32 bands of 32 columns
__host__ __device__ __forceinline__ int hpad(int i) { return i + (i >> 5); }

size_t diff_hT_smem(int X, int wx)
{
    const int seg = min(X, kHSeg), span = seg + 2 * wx;
    return (size_t)(kDC + 1) * hpad(span + 31) * 4 + (size_t)kDiffNT * 33 * 4;
}

__global__ void __launch_bounds__(kDiffNT) diff_hT_kernel(const float *__restrict__ g1,
                                                          const uint32_t *__restrict__ arm, int X, int Y, int wx,
                                                          int dc, float *__restrict__ g2)
{
    extern __shared__ float hsm[];
    const int seg = min(X, kHSeg), span = seg + 2 * wx, pitch = hpad(span + 31);
    float *gs = hsm;                                          // [kDC][pitch] staged planes, then outputs
    uint32_t *as = reinterpret_cast<uint32_t *>(hsm + kDC * pitch);   // [pitch] arm words
    float *delta = hsm + (kDC + 1) * pitch;                   // [kDiffNT][33]
    const int y = blockIdx.y, x0 = blockIdx.x * kHSeg;
    const int xs = x0 - wx;                                   // column of staged index 0
    const int x1 = min(x0 + kHSeg, X);                        // segment columns [x0, x1)
    const size_t b = blockIdx.z, n = (size_t)X * Y;           // pair
    const size_t r = (size_t)y * X;
    g1 += b * kDC * n;
    g2 += b * kDC * n;
    arm += b * n;
    // stage the planes and arms of columns [max(xs, 0), min(x1 + wx, X))
    const int sa = max(xs, 0), sb = min(x1 + wx, X);
    for (int x = sa + (int)threadIdx.x; x < sb; x += kDiffNT) {
        as[hpad(x - xs)] = arm[r + x];
        for (int k = 0; k < dc; ++k) gs[k * pitch + hpad(x - xs)] = g1[(size_t)k * n + r + x];
    }
    __syncthreads();
    const int k = threadIdx.x / 32, band = threadIdx.x % 32;
    const int bx0 = x0 + 32 * band;                           // band columns [bx0, be)
    const int be = min(bx0 + 32, x1);
    float *dl = delta + threadIdx.x * 33;
    float acc[32];
    const bool work = k < dc && bx0 < be;
    if (work) {
#pragma unroll
        for (int i = 0; i <= 32; ++i) dl[i] = 0.f;
        const float *gk = gs + k * pitch;
        const int xa = max(bx0 - wx, 0), xb = min(be - 1 + wx, X - 1);
        for (int x = xa; x <= xb; ++x) {
            const uint32_t am = as[hpad(x - xs)];
            const int lo = x - (int)(am & 0xFF), hi = x + (int)((am >> 8) & 0xFF);
            if (hi < bx0 || lo >= be) continue;
            const float v = gk[hpad(x - xs)];
            dl[max(lo, bx0) - bx0] += v;
            if (hi + 1 < be) dl[hi + 1 - bx0] -= v;
        }
        float sacc = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            sacc += dl[i];
            acc[i] = sacc;
        }
    }
    __syncthreads();                              // every thread is done with the staged planes
    if (work)
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (bx0 + i < be) gs[k * pitch + hpad(bx0 + i - xs)] = acc[i];
    __syncthreads();
    for (int x = x0 + (int)threadIdx.x; x < x1; x += kDiffNT)
        for (int kk = 0; kk < dc; ++kk) g2[(size_t)kk * n + r + x] = gs[kk * pitch + hpad(x - xs)];
}

// Backward 4: through the cost. Per pixel: its own gradient as the left pixel
// of every cell (x, y, d), as the right pixel x' of the cells (x' + d, y, d),
// and its cells' contributions to the four parameters (one partial per block,
// summed later in a fixed order).
__global__ void diff_costgrad_kernel(const float *__restrict__ gL, const float *__restrict__ gR,
                                     const uint32_t *__restrict__ pixL, const uint32_t *__restrict__ pixR,
                                     const float *__restrict__ theta, int X, int Y, int D, int d0, int dc,
                                     const float *__restrict__ g2, float *__restrict__ acc_l,
                                     float *__restrict__ acc_r, float *__restrict__ part, size_t part_pair)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t b = blockIdx.y, n = (size_t)X * Y;   // pair
    gL += b * n;
    gR += b * n;
    pixL += b * n;
    pixR += b * n;
    g2 += b * kDC * n;
    acc_l += b * n;
    acc_r += b * n;
    part += b * part_pair;
    const Theta th = load_theta(theta);
    const float inv_lad = 1.f / th.lad, inv_lmc = 1.f / th.lmc;
    const float kad = th.wad * inv_lad;                 // w_AD / l_AD
    const float dad = th.wad * inv_lad * inv_lad;       // w_AD / l_AD^2
    const float dmc = th.wmc * inv_lmc * inv_lmc;       // w_MC / l_MC^2
    // exp(-h / l_MC) for the seven Hamming distances
    __shared__ float eh_t[8];
    if (threadIdx.x < 7) eh_t[threadIdx.x] = expf(-(float)threadIdx.x * inv_lmc);
    __syncthreads();
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
    if (i < X * Y) {
        const int y = i / X, x = i - y * X;
        const size_t r = (size_t)y * X;
        const int kn = min(dc, D - d0);
        const float gl = gL[i], gr = gR[i];
        const uint32_t pl = pixL[i];
        const float ea1 = expf(-inv_lad), eh6 = eh_t[6];   // the terms of P (|a| = 1, h = 6)
        float al = 0.f, ar = 0.f;
        // the chunk's disparities unrolled, so their loads and exps overlap
#pragma unroll
        for (int k = 0; k < kDC; ++k) {
            if (k < kn) {
                const int d = d0 + k;
                const float *plane = g2 + (size_t)k * X * Y;
                const float g = plane[i];
                if (x < d) {
                    t0 += g * (1.f - ea1);
                    t1 += g * (1.f - eh6);
                    t2 += g * (-ea1 * dad);
                    t3 += g * (-eh6 * 6.f * dmc);
                } else {
                    const float diff = gl - gR[i - d], a = fabsf(diff);
                    const int hi = __popc((pl ^ pixR[i - d]) & 0x3F00u);
                    const float h = (float)hi;
                    const float ea = expf(-a * inv_lad), eh = eh_t[hi];
                    t0 += g * (1.f - ea);
                    t1 += g * (1.f - eh);
                    t2 += g * (-ea * a * dad);
                    t3 += g * (-eh * h * dmc);
                    const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
                    al += g * kad * ea * sgn;
                }
                // this pixel as the match of the left pixel x + d
                if (x + d < X) {
                    const float gg = plane[r + x + d];
                    const float diff = gL[r + x + d] - gr, a = fabsf(diff);
                    const float ea = expf(-a * inv_lad);
                    const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
                    ar -= gg * kad * ea * sgn;
                }
            }
        }
        acc_l[i] += al;
        acc_r[i] += ar;
    }
    // block partials of the parameter gradients
    __shared__ float sh[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_down_sync(0xffffffffu, t0, o);
        t1 += __shfl_down_sync(0xffffffffu, t1, o);
        t2 += __shfl_down_sync(0xffffffffu, t2, o);
        t3 += __shfl_down_sync(0xffffffffu, t3, o);
    }
    if (lane == 0) {
        sh[0][w] = t0;
        sh[1][w] = t1;
        sh[2][w] = t2;
        sh[3][w] = t3;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float s = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[threadIdx.x][k];
        part[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
    }
}

__global__ void diff_finish_kernel(const float *__restrict__ acc_l, const float *__restrict__ acc_r, int n,
                                   float *__restrict__ grad_l, float *__restrict__ grad_r)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t b = blockIdx.y;                  // pair
    acc_l += b * n;
    acc_r += b * n;
    grad_l += b * n * 3;
    grad_r += b * n * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        grad_l[3 * i + c] = acc_l[i] * kGreyW[c];
        grad_r[3 * i + c] = acc_r[i] * kGreyW[c];
    }
}

// Sum of all block partials in a fixed order (double accumulation), in two
// levels so that the FP64 adds spread over the GPU. Level 1: block j sums the
// contiguous segment j of the partials (thread t takes its elements t, t +
// kRedNT, ... in turn, then a fixed pairwise tree adds the threads' sums).
// Level 2: one block adds the kRedBlocks segment sums by the same fixed tree.
// Neither order depends on scheduling.
constexpr int kRedNT = 256;
constexpr int kRedBlocks = 128;

__device__ __forceinline__ void tree_sum4(double (*sh)[kRedNT], double s0, double s1, double s2, double s3)
{
    const int t = threadIdx.x;
    sh[0][t] = s0;
    sh[1][t] = s1;
    sh[2][t] = s2;
    sh[3][t] = s3;
    __syncthreads();
    for (int o = kRedNT / 2; o > 0; o >>= 1) {
        if (t < o)
#pragma unroll
            for (int c = 0; c < 4; ++c) sh[c][t] += sh[c][t + o];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kRedNT) diff_theta_segments_kernel(const float *__restrict__ part, int nparts,
                                                                     double *__restrict__ seg)
{
    __shared__ double sh[4][kRedNT];
    const int t = threadIdx.x, len = (nparts + kRedBlocks - 1) / kRedBlocks;
    const int k0 = min(nparts, (int)blockIdx.x * len), k1 = min(nparts, k0 + len);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int k = k0 + t; k < k1; k += kRedNT) {
        const float4 v = *reinterpret_cast<const float4 *>(part + (size_t)k * 4);
        s0 += (double)v.x;
        s1 += (double)v.y;
        s2 += (double)v.z;
        s3 += (double)v.w;
    }
    tree_sum4(sh, s0, s1, s2, s3);
    if (t < 4) seg[blockIdx.x * 4 + t] = sh[t][0];
}

__global__ void __launch_bounds__(kRedNT) diff_theta_reduce_kernel(const double *__restrict__ seg,
                                                                   float *__restrict__ grad)
{
    static_assert(kRedBlocks <= kRedNT, "one segment sum per thread");
    __shared__ double sh[4][kRedNT];
    const int t = threadIdx.x;
    const bool h = t < kRedBlocks;
    tree_sum4(sh, h ? seg[t * 4] : 0.0, h ? seg[t * 4 + 1] : 0.0, h ? seg[t * 4 + 2] : 0.0, h ? seg[t * 4 + 3] : 0.0);
    if (t < 4) grad[t] = (float)sh[t][0];
}

}  // namespace

// Workspace of a batch: per-pair planes [B][...] of each kind, then the
// parameter-gradient partials [B][chunk][block][4]. With base == nullptr
// only the size is computed.
struct DiffWs {
    float *gl, *gr;
    uint8_t *ql, *qr;
    uint32_t *pixl, *pixr, *arml, *armr, *armcl, *armcr, *keyl, *keyr;
    float *ns, *state, *accl, *accr, *s0, *s1, *s2, *s3, *part;
    double *seg;
};

size_t diff_layout(char *base, int X, int Y, int wy, int B, int D, DiffWs *w)
{
    const size_t n = (size_t)X * Y, nb = (size_t)B;
    const size_t nblk = (n + kDiffNT - 1) / kDiffNT;
    const size_t nchunks = (D + kDC - 1) / kDC;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    DiffWs t;
    t.gl = (float *)take(nb * n * 4);                        // float grey
    t.gr = (float *)take(nb * n * 4);
    t.ql = (uint8_t *)take(nb * n);                          // integer grey of the uint8 images
    t.qr = (uint8_t *)take(nb * n);
    t.pixl = (uint32_t *)take(nb * n * 4);                   // pixel and arm words
    t.pixr = (uint32_t *)take(nb * n * 4);
    t.arml = (uint32_t *)take(nb * n * 4);
    t.armr = (uint32_t *)take(nb * n * 4);
    t.armcl = (uint32_t *)take(nb * armc_words(X, Y, wy) * 4);
    t.armcr = (uint32_t *)take(nb * armc_words(X, Y, wy) * 4);
    t.keyl = (uint32_t *)take(nb * n * 4);                   // keys (written by the support pass)
    t.keyr = (uint32_t *)take(nb * n * 4);
    t.ns = (float *)take(nb * n * 4);                        // support size
    t.state = (float *)take(nb * n * 4 * 3);                 // online softmax state
    t.accl = (float *)take(nb * n * 4);                      // intensity-gradient accumulators
    t.accr = (float *)take(nb * n * 4);
    t.s0 = (float *)take(nb * kDC * n * 4);                  // slabs
    t.s1 = (float *)take(nb * kDC * n * 4);
    t.s2 = (float *)take(nb * kDC * n * 4);
    t.s3 = (float *)take(nb * kDC * n * 4);
    t.part = (float *)take(nb * nchunks * nblk * 16);        // parameter-gradient partials
    t.seg = (double *)take(kRedBlocks * 4 * sizeof(double)); // their segment sums
    if (w) *w = t;
    return off;
}

size_t diff_workspace_bytes(int X, int Y, int wy, int B, int D)
{
    return diff_layout(nullptr, X, Y, wy, B, D, nullptr);
}

cudaError_t diff_setup()
{
    // the cost rows of a chunk take up to kDC * 4096 floats of shared memory;
    // the horizontal adjoint stages a 1024-column segment with a halo of up to
    // 141 columns each side
    cudaError_t e = cudaFuncSetAttribute(diff_costx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kDC * 4096 * (int)sizeof(float));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(diff_hT_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)diff_hT_smem(kHSeg, kMaxWx));
}

cudaError_t diff_run(const DiffArgs &a, cudaStream_t s)
{
    const int X = a.W, Y = a.H, n = X * Y, B = a.B;
    DiffWs w;
    diff_layout((char *)a.ws, X, Y, a.wy, B, a.D, &w);
    const int nblk = (n + kDiffNT - 1) / kDiffNT;
    const int nchunks = (a.D + kDC - 1) / kDC;
    const size_t part_pair = (size_t)nchunks * nblk * 4;
    const size_t armc_n = armc_words(X, Y, a.wy);
    const float inv_tau = 1.f / a.tau;
    const dim3 tiles((X + kTileX - 1) / kTileX, (Y + kTileY - 1) / kTileY, B);
    static_assert(kTileX * kTileY == kDiffNT, "one thread per pixel of a tile");
    cudaError_t e = cudaSuccess;
    // frozen supports of every pair (integer path), support sizes, float grey
    diff_grey_kernel<<<dim3(nblk, 2, B), kDiffNT, 0, s>>>(a.left, a.right, w.gl, w.gr, n);
    for (int b = 0; b < B; ++b) {
        const size_t o = (size_t)b * n;
        if ((e = launch_grey(a.left_u8 + o * 3, a.right_u8 + o * 3, w.ql + o, w.qr + o, X, Y, s)) != cudaSuccess ||
            (e = launch_support(w.ql + o, w.qr + o, w.pixl + o, w.pixr + o, w.arml + o, w.armr + o,
                                w.armcl + b * armc_n, w.armcr + b * armc_n, w.keyl + o, w.keyr + o, a.err, X, Y,
                                a.wx, a.wy, a.tc, s)) != cudaSuccess)
            return e;
    }
    diff_nsupport_kernel<<<dim3(nblk, B), kDiffNT, 0, s>>>(w.arml, X, Y, w.ns);
    if (a.backward) {
        if ((e = cudaMemsetAsync(w.accl, 0, (size_t)B * n * 4, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(w.accr, 0, (size_t)B * n * 4, s)) != cudaSuccess)
            return e;
    }
    for (int c = 0; c < nchunks; ++c) {
        const int d0 = c * kDC, dc = min(kDC, a.D - d0);
        diff_costx_kernel<<<dim3(Y, B), kDiffNT, (size_t)dc * X * 4, s>>>(w.gl, w.gr, w.pixl, w.pixr, w.arml,
                                                                          a.theta, X, Y, a.D, d0, dc, w.s0);
        if (!a.backward) {
            diff_vagg_softmax_kernel<<<tiles, kDiffNT, 0, s>>>(w.s0, w.arml, w.ns, X, Y, a.D, d0, dc,
                                                                       inv_tau, w.state, c == 0, c == nchunks - 1,
                                                                       a.dhat, a.stats);
        } else {
            diff_gca_kernel<<<tiles, kDiffNT, 0, s>>>(w.s0, w.arml, w.ns, X, Y, a.D, d0, dc, inv_tau,
                                                              a.dhat, a.stats, a.grad_dhat, w.s1);
            diff_vT_kernel<<<dim3((X + 31) / 32, (Y + kVB - 1) / kVB, B), kDiffNT, 0, s>>>(w.s1, w.arml, X, Y,
                                                                                      a.wy, dc, w.s2);
            diff_hT_kernel<<<dim3((X + kHSeg - 1) / kHSeg, Y, B), kDiffNT, diff_hT_smem(X, a.wx), s>>>(
                w.s2, w.arml, X, Y, a.wx, dc, w.s3);
            diff_costgrad_kernel<<<dim3(nblk, B), kDiffNT, 0, s>>>(w.gl, w.gr, w.pixl, w.pixr, a.theta, X, Y, a.D,
                                                                   d0, dc, w.s3, w.accl, w.accr,
                                                                   w.part + (size_t)c * nblk * 4, part_pair);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.backward) {
        diff_finish_kernel<<<dim3(nblk, B), kDiffNT, 0, s>>>(w.accl, w.accr, n, a.grad_left, a.grad_right);
        diff_theta_segments_kernel<<<kRedBlocks, kRedNT, 0, s>>>(w.part, B * nchunks * nblk, w.seg);
        diff_theta_reduce_kernel<<<1, kRedNT, 0, s>>>(w.seg, a.grad_theta);
    }
    return cudaGetLastError();
}

}  // namespace stereo
