// Preprocessing kernels: grey conversion (Sec. III step 1), 2x mean-pool
// downscale (Sec. III-A, Eq. 2), and the per-pixel support data of the fused
// kernel: mini-census code (Sec. III-B) and the four cross arms (Sec. III-C).
// These are short passes over a few MB: each pixel is read from HBM once,
// the grey + downscale pass keeps its neighbourhoods in registers and the
// support pass stages them in shared memory.
#include "internal.cuh"

namespace stereo {
namespace {

__device__ __forceinline__ uint32_t luma(uint32_t r, uint32_t g, uint32_t b)
{
    // Step 1 gives no formula: BT.601 weights in 8-bit fixed point, rounded.
    return (77u * r + 150u * g + 29u * b + 128u) >> 8;
}

// The weights of luma() as the bytes of one word (r in byte 0).
constexpr uint32_t kLumaW = 77u | (150u << 8) | (29u << 16);

// luma() of the four pixels in three aligned words (w0 = r0 g0 b0 r1, w1 =
// g1 b1 r2 g2, w2 = b2 r3 g3 b3), packed one grey byte per pixel: each
// weighted sum is a four-byte dot product of the pixel's (r, g, b, -) bytes
// with (77, 150, 29, 0), and its byte 1 is the grey value (sum >> 8).
__device__ __forceinline__ uint32_t luma4(uint32_t w0, uint32_t w1, uint32_t w2)
{
    const uint32_t l0 = __dp4a(w0, kLumaW, 128u);
    const uint32_t l1 = __dp4a(__funnelshift_r(w0, w1, 24), kLumaW, 128u);
    const uint32_t l2 = __dp4a(__funnelshift_r(w1, w2, 16), kLumaW, 128u);
    const uint32_t l3 = __dp4a(w2, kLumaW << 8, 128u);
    return __byte_perm(__byte_perm(l0, l1, 0x5151), __byte_perm(l2, l3, 0x5151), 0x5410);
}

// RGB (HWC) -> grey for both images (blockIdx.y selects the image). Each
// thread converts four consecutive pixels; with a 4-byte aligned source those
// twelve bytes are three aligned 32-bit loads.
template <bool kAligned>
__global__ void grey_kernel(const uint8_t *__restrict__ rgb_l, const uint8_t *__restrict__ rgb_r,
                            uint8_t *__restrict__ g_l, uint8_t *__restrict__ g_r, long n)
{
    const uint8_t *rgb = blockIdx.y ? rgb_r : rgb_l;
    uint8_t *g = blockIdx.y ? g_r : g_l;
    long p = 4 * ((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (p >= n) return;
    if (kAligned && p + 4 <= n) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(rgb + 3 * p);
        *reinterpret_cast<uint32_t *>(g + p) = luma4(__ldg(w), __ldg(w + 1), __ldg(w + 2));
    } else {
        for (long q = p; q < p + 4 && q < n; ++q)
            g[q] = (uint8_t)luma(rgb[3 * q], rgb[3 * q + 1], rgb[3 * q + 2]);
    }
}

// Eq. 2 with K = 2, m = 1: mean of the 3x3 window centred on (2x, 2y),
// coordinates clamped to the image, rounded half up: (sum + 4) / 9.
__global__ void downscale_kernel(const uint8_t *__restrict__ g_l, const uint8_t *__restrict__ g_r,
                                 uint8_t *__restrict__ s_l, uint8_t *__restrict__ s_r, int W, int H)
{
    const uint8_t *g = blockIdx.z ? g_r : g_l;
    uint8_t *s = blockIdx.z ? s_r : s_l;
    int X = W / 2, Y = H / 2;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= X || y >= Y) return;
    int sum = 0;
#pragma unroll
    for (int j = -1; j <= 1; ++j) {
        int yy = min(max(2 * y + j, 0), H - 1);
        const uint8_t *row = g + (size_t)yy * W;
#pragma unroll
        for (int i = -1; i <= 1; ++i) sum += __ldg(row + min(max(2 * x + i, 0), W - 1));
    }
    s[(size_t)y * X + x] = (uint8_t)((sum + 4) / 9);
}

// Grey conversion and Eq. 2 downscale in one pass (the downscaling path, for
// W a multiple of 4 and 4-byte aligned RGB rows). Thread (band, c) of one
// image owns full-res columns 4c .. 4c + 3 and makes the 3x3 means of output
// columns 2c, 2c + 1, rows 4 band .. 4 band + 3. It converts rows
// 8 band - 1 .. 8 band + 7 of its columns (row coordinates clamped, as in
// downscale_kernel), each from three aligned words, all requested before the
// first is used; the grey of pixel 4c - 1 comes from the word its left
// neighbour loaded (a shuffle; lane 0 loads it itself). Grey values stay in
// registers; the left image's full-res grey of rows 8 band .. 8 band + 7 is
// written for the scale-up. Bands cover ceil(H / 2) rows so that the last row
// of an odd H gets its grey. Same arithmetic as grey_kernel followed by
// downscale_kernel.
constexpr int kGDT = 128;                  // threads per CTA
constexpr int kGDB = 4;                    // output rows per thread
constexpr int kGDR = 2 * kGDB + 1;         // full-res rows per thread

__global__ void __launch_bounds__(kGDT) grey_down_kernel(
    const uint8_t *__restrict__ rgb_l, const uint8_t *__restrict__ rgb_r, uint8_t *__restrict__ gf_l,
    uint8_t *__restrict__ s_l, uint8_t *__restrict__ s_r, int W, int H, int ncol, int nband)
{
    pdl_trigger();
    pdl_wait();   // launched early behind the previous frame's last kernel, which still reads gf and s
    const bool right = blockIdx.y != 0;
    const int t0 = blockIdx.x * kGDT + threadIdx.x;
    const int nthr = ncol * nband;
    // threads past the end take the last thread's pixels for the shuffles
    // and store nothing
    const bool live = t0 < nthr;
    const int t = live ? t0 : nthr - 1;
    const int band = t / ncol, c = t - band * ncol;   // left neighbour (band, c - 1) is thread t - 1
    const int lane = threadIdx.x & 31;
    const uint8_t *rgb = right ? rgb_r : rgb_l;
    uint8_t *s = right ? s_r : s_l;
    const int X = W / 2, Y = H / 2;
    uint32_t w[kGDR][3], wh[kGDR];
#pragma unroll
    for (int r = 0; r < kGDR; ++r) {
        const int fy = min(max(8 * band - 1 + r, 0), H - 1);
        const uint32_t *p = reinterpret_cast<const uint32_t *>(rgb + ((size_t)fy * W + 4 * c) * 3);
#pragma unroll
        for (int i = 0; i < 3; ++i) w[r][i] = __ldg(p + i);
        wh[r] = lane == 0 && c > 0 ? __ldg(p - 1) : 0u;
    }
    // horizontal 3-sums of row r at full-res columns 4c and 4c + 2
    uint32_t hs[kGDR][2];
#pragma unroll
    for (int r = 0; r < kGDR; ++r) {
        // the word before this thread's first: pixel 4c - 1 in bytes 1..3
        const uint32_t prev = __shfl_up_sync(0xffffffffu, w[r][2], 1);
        const uint32_t hw = lane == 0 ? wh[r] : prev;
        const uint32_t g = luma4(w[r][0], w[r][1], w[r][2]);
        // pixel 4c - 1, or pixel 0 (clamped) for the first column group
        const uint32_t gh = c > 0 ? __dp4a(hw, kLumaW << 8, 128u) >> 8 : (g & 0xFFu);
        hs[r][0] = __dp4a(g, 0x00000101u, gh);
        hs[r][1] = __dp4a(g, 0x01010100u, 0u);
        const int fy = 8 * band - 1 + r;
        if (live && !right && r > 0 && fy < H) *reinterpret_cast<uint32_t *>(gf_l + (size_t)fy * W + 4 * c) = g;
    }
    if (!live) return;
#pragma unroll
    for (int i = 0; i < kGDB; ++i) {
        const int y = kGDB * band + i;
        if (y >= Y) break;
        const uint32_t m0 = (hs[2 * i][0] + hs[2 * i + 1][0] + hs[2 * i + 2][0] + 4u) / 9u;
        const uint32_t m1 = (hs[2 * i][1] + hs[2 * i + 1][1] + hs[2 * i + 2][1] + 4u) / 9u;
        // X is even: output pixel 2c starts a 2-byte aligned pair
        *reinterpret_cast<uint16_t *>(s + (size_t)y * X + 2 * c) = (uint16_t)(m0 | m1 << 8);
    }
}

// Support data in two passes, each with a halo only along its own axis.
//  Pass H: rows of kHX pixels (plus wx + 7 pixels each side and one row
//  above and below): census code and left/right arms; grey | census << 8 goes
//  to the pixel word, the left/right arms to the low half of the arm words.
//  Pass V: columns of kVY pixels (plus kMaxWy + 7 rows above and below): up/down
//  arms to the high half of the arm words.
// Coordinates of the staged tiles are clamped to the image (border
// replication, which census reads); the arm scans stop at the real border.
//
// Arm length from the staged pixel t (value c) in direction DIR (+1 or -1,
// element stride S): the number of consecutive pixels k = 1, 2, ... with
// |I - c| < tc, at most cap (Sec. III-C). Pixels are tested in chunks of
// kArmChunk; the tile holds kArmChunk - 1 pixels beyond each cap. Arm lengths
// vary a lot between neighbouring pixels, so a warp whose lanes each follow
// their own arm to its end idles most lanes while the longest arm finishes.
// Instead every thread tests the first chunk of each of its arms; the arms
// that go on are appended to a per-CTA queue, and the threads then take
// queued arms in turn, one chunk per step, each lane moving to its next arm
// as soon as one ends, so the lanes stay busy until the queue is drained.
constexpr int kArmChunk = 8;
constexpr int kSupNT = 256;                   // threads of a support CTA

// Similar pixels at the head of a chunk of N pixels from p (element step
// DIR * S).
template <int DIR, int S, int N>
__device__ __forceinline__ int arm_chunk(const uint8_t *p, int off, unsigned lim)
{
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) m |= (uint32_t)((unsigned)(p[DIR * j * S] + off) < lim) << j;
    return __ffs(~m) - 1;
}

// The same with a step known only at run time (queued arms of both
// directions).
__device__ __forceinline__ int arm_chunk_dyn(const uint8_t *p, int step, int off, unsigned lim)
{
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < kArmChunk; ++j) m |= (uint32_t)((unsigned)(p[j * step] + off) < lim) << j;
    return __ffs(~m) - 1;
}

// |I - c| < tc  <=>  (unsigned)(I - c + tc - 1) < 2 tc - 1; tc = 0: nothing
// is similar.
__device__ __forceinline__ unsigned arm_lim(int tc)
{
    return tc > 0 ? (unsigned)(2 * tc - 1) : 0u;
}

// Queue entry of an arm that goes on past its first chunk: the pixel's
// offset in the tile (12 bits), its output slot (11 bits), the direction
// (1 bit: 0 towards lower coordinates) and the cap (8 bits).
__device__ __forceinline__ uint32_t arm_entry(int toff, int slot, int dir, int cap)
{
    return (uint32_t)toff | ((uint32_t)slot << 12) | ((uint32_t)dir << 23) | ((uint32_t)cap << 24);
}

// First chunk of an arm; `more` is set when the arm may go on.
template <int DIR, int S>
__device__ __forceinline__ int arm_first(const uint8_t *t, int off, unsigned lim, int cap, bool &more)
{
    const int run = arm_chunk<DIR, S, kArmChunk>(t + DIR * S, off, lim);
    const int n = min(run, cap);
    more = run == kArmChunk && n < cap;
    return n;
}

// Appends this thread's queued arms (e[j] where bit j of `more` is set).
template <int N>
__device__ __forceinline__ void arm_push(uint32_t *q, int *nq, const uint32_t (&e)[N], uint32_t more)
{
    if (more == 0u) return;
    int w = atomicAdd(nq, __popc(more));
#pragma unroll
    for (int j = 0; j < N; ++j)
        if ((more >> j) & 1u) q[w++] = e[j];
}

// Drains the queue: each thread takes entries threadIdx.x, + kSupNT, ...,
// one chunk per step, and writes each arm's length to res[dir][slot].
__device__ __forceinline__ void arm_drain(const uint8_t *tile, const uint32_t *q, int nq, uint8_t *res,
                                          int nslot, int S, int tc)
{
    const unsigned lim = arm_lim(tc);
    int i = threadIdx.x;
    const uint8_t *p = tile;
    int step = 0, off = 0, cap = 0, n = 0, slot = 0, dir = 0;
    auto setup = [&](uint32_t e) {
        p = tile + (e & 0xFFFu);
        slot = (e >> 12) & 0x7FF;
        dir = (e >> 23) & 1;
        cap = (int)(e >> 24);
        step = dir ? S : -S;
        off = tc - 1 - (int)p[0];
        n = kArmChunk;                            // the first chunk was all similar
    };
    bool have = i < nq;
    if (have) setup(q[i]);
    while (have) {
        const int run = arm_chunk_dyn(p + step * (n + 1), step, off, lim);
        n = min(n + run, cap);
        if (run < kArmChunk || n >= cap) {
            res[dir * nslot + slot] = (uint8_t)n;
            i += kSupNT;
            have = i < nq;
            if (have) setup(q[i]);
        }
    }
}

constexpr int kHX = 256;   // pass H: outputs per row tile (one column per thread)
constexpr int kHY = 4;     // pass H: rows per CTA
constexpr int kVX = 32;    // pass V: columns per CTA
constexpr int kVY = 16;    // pass V: outputs per column tile
constexpr int kHXH = kMaxWx + kArmChunk - 1;   // pass H halo at the largest cap (wx + 7 at run time)
constexpr int kVYH = kMaxWy + kArmChunk - 1;   // pass V halo
static_assert(kHX == kSupNT, "pass H: one column per thread");
static_assert(kSupNT % kVX == 0 && kVY % (kSupNT / kVX) == 0, "pass V: whole rows per thread");
static_assert((kHX + 2 * kHXH) * (kHY + 2) < 4096 && kVX * (kVY + 2 * kVYH) < 4096, "tile offsets take 12 bits");
static_assert(kHY * kHX <= 2048 && kVY * kVX <= 2048, "output slots take 11 bits");
static_assert(kMaxWx < 256 && kMaxWy < 256, "caps take 8 bits");

// Shared memory of one pass: tile, arm lengths [2][slots], queue [2 * slots], count.
__host__ __device__ constexpr int sup_tile_bytes(int tile, int slots)
{
    return (tile + 15) / 16 * 16 + 2 * slots + 4 * 2 * slots + 16;
}
constexpr int kSupSmemH = sup_tile_bytes((kHX + 2 * kHXH) * (kHY + 2), kHY * kHX);
constexpr int kSupSmemV = sup_tile_bytes(kVX * (kVY + 2 * kVYH), kVY * kVX);

struct SupportArgs {
    const uint8_t *g_l, *g_r;
    uint32_t *pix_l, *pix_r, *arm_l, *arm_r, *armc_l, *armc_r, *key_l, *key_r, *err;
    int X, Y, wx, wy, tc;
    int nhx, nhy, nvx, nvy;                       // tiles of pass H and pass V per image
};

// Pass H on row tile (bx, by) of image bz.
__device__ __forceinline__ void support_h(const SupportArgs &A, uint8_t *smem, int bx, int by, int bz)
{
    const int X = A.X, Y = A.Y, wx = A.wx, tc = A.tc;
    const uint8_t *g = bz ? A.g_r : A.g_l;
    uint32_t *pix = bz ? A.pix_r : A.pix_l;
    uint16_t *arm = reinterpret_cast<uint16_t *>(bz ? A.arm_r : A.arm_l);
    uint16_t *armc = reinterpret_cast<uint16_t *>(bz ? A.armc_r : A.armc_l);
    uint32_t *key = bz ? A.key_r : A.key_l;
    // the staged row holds the tile's pixels and wx + 7 more on each side
    // (the first chunk of an arm at its cap reads 7 beyond it; >= 2 for census)
    const int hx = wx + kArmChunk - 1, TW = kHX + 2 * hx;
    constexpr int TH = kHY + 2, NS = kHY * kHX;
    uint8_t *tile = smem;
    uint8_t *res = smem + ((kHX + 2 * kHXH) * TH + 15) / 16 * 16;   // [2][NS]
    uint32_t *q = reinterpret_cast<uint32_t *>(res + 2 * NS);       // [2 NS]
    int *nq = reinterpret_cast<int *>(q + 2 * NS);
    const int x0 = bx * kHX, y0 = by * kHY;
    if ((bx | by | bz | threadIdx.x) == 0) *A.err = 0u;
    if (threadIdx.x == 0) *nq = 0;

    for (int ty = 0; ty < TH; ++ty) {
        const uint8_t *row = g + (size_t)min(max(y0 - 1 + ty, 0), Y - 1) * X;
        for (int tx = threadIdx.x; tx < TW; tx += kSupNT)
            tile[ty * TW + tx] = __ldg(row + min(max(x0 - hx + tx, 0), X - 1));
    }
    __syncthreads();

    // Census pattern (Fig. 3 is missing): six neighbours in rows y-1..y+1,
    // mirror-symmetric in x; bit k set when neighbour k is strictly darker.
    const int cdx[6] = {-1, +1, -2, +2, -1, +1};
    const int cdy[6] = {-1, -1, 0, 0, +1, +1};
    const unsigned lim = arm_lim(tc);
    const int ox = threadIdx.x, x = x0 + ox;
    uint32_t e[2 * kHY], more = 0;
#pragma unroll
    for (int oy = 0; oy < kHY; ++oy) {
        const int y = y0 + oy;
        const bool valid = x < X && y < Y;
        const int toff = (oy + 1) * TW + ox + hx;
        const uint8_t *t = tile + toff;
        const int c = t[0];
        uint32_t code = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) code |= (uint32_t)(t[cdy[k] * TW + cdx[k]] < c) << k;
        const int off = tc - 1 - c;
        const int cm = valid ? min(wx, x) : 0, cp = valid ? min(wx, X - 1 - x) : 0;
        bool mm, mp;
        const int slot = oy * kHX + ox;
        res[slot] = (uint8_t)arm_first<-1, 1>(t, off, lim, cm, mm);
        res[NS + slot] = (uint8_t)arm_first<1, 1>(t, off, lim, cp, mp);
        e[2 * oy] = arm_entry(toff, slot, 0, cm);
        e[2 * oy + 1] = arm_entry(toff, slot, 1, cp);
        more |= ((uint32_t)mm << (2 * oy)) | ((uint32_t)mp << (2 * oy + 1));
        if (valid) {
            const size_t idx = (size_t)y * X + x;
            pix[idx] = (uint32_t)c | (code << 8);
            key[idx] = 0xFFFFFFFFu;               // WTA key preset: the fused kernel takes atomic minima
        }
    }
    arm_push(q, nq, e, more);
    __syncthreads();
    arm_drain(tile, q, *nq, res, NS, 1, tc);
    __syncthreads();
#pragma unroll
    for (int oy = 0; oy < kHY; ++oy) {
        const int y = y0 + oy, slot = oy * kHX + ox;
        if (x < X && y < Y) {
            const size_t idx = (size_t)y * X + x;
            const uint16_t h = (uint16_t)(res[slot] | (res[NS + slot] << 8));
            arm[2 * idx] = h;
            armc[2 * armc_index(y, x, X)] = h;   // the fused kernel reads row y's left/right arms in row y
        }
    }
}

// Pass V on column tile (bx, by) of image bz.
__device__ __forceinline__ void support_v(const SupportArgs &A, uint8_t *smem, int bx, int by, int bz)
{
    const int X = A.X, Y = A.Y, wy = A.wy, tc = A.tc;
    const uint8_t *g = bz ? A.g_r : A.g_l;
    uint16_t *arm = reinterpret_cast<uint16_t *>(bz ? A.arm_r : A.arm_l);
    uint16_t *armc = reinterpret_cast<uint16_t *>(bz ? A.armc_r : A.armc_l);
    constexpr int hy = kVYH, TH = kVY + 2 * hy, NS = kVY * kVX, RPT = kVY / (kSupNT / kVX);
    uint8_t *tile = smem;
    uint8_t *res = smem + (kVX * TH + 15) / 16 * 16;            // [2][NS]
    uint32_t *q = reinterpret_cast<uint32_t *>(res + 2 * NS);   // [2 NS]
    int *nq = reinterpret_cast<int *>(q + 2 * NS);
    const int x0 = bx * kVX, y0 = by * kVY;
    const int tx = threadIdx.x % kVX, tq = threadIdx.x / kVX;     // kSupNT / kVX threads per column
    const int x = min(x0 + tx, X - 1);
    if (threadIdx.x == 0) *nq = 0;
    for (int ty = tq; ty < TH; ty += kSupNT / kVX)
        tile[ty * kVX + tx] = __ldg(g + (size_t)min(max(y0 - hy + ty, 0), Y - 1) * X + x);
    __syncthreads();
    const unsigned lim = arm_lim(tc);
    uint32_t e[2 * RPT], more = 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int oy = tq + r * (kSupNT / kVX), y = y0 + oy;
        const bool valid = x0 + tx < X && y < Y;
        const int toff = (oy + hy) * kVX + tx;
        const uint8_t *t = tile + toff;
        const int off = tc - 1 - (int)t[0];
        const int cm = valid ? min(wy, y) : 0, cp = valid ? min(wy, Y - 1 - y) : 0;
        bool mm, mp;
        const int slot = oy * kVX + tx;
        res[slot] = (uint8_t)arm_first<-1, kVX>(t, off, lim, cm, mm);
        res[NS + slot] = (uint8_t)arm_first<1, kVX>(t, off, lim, cp, mp);
        e[2 * r] = arm_entry(toff, slot, 0, cm);
        e[2 * r + 1] = arm_entry(toff, slot, 1, cp);
        more |= ((uint32_t)mm << (2 * r)) | ((uint32_t)mp << (2 * r + 1));
    }
    arm_push(q, nq, e, more);
    __syncthreads();
    arm_drain(tile, q, *nq, res, NS, kVX, tc);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int oy = tq + r * (kSupNT / kVX), y = y0 + oy, slot = oy * kVX + tx;
        if (x0 + tx < X && y < Y) {
            const uint16_t v = (uint16_t)(res[slot] | (res[NS + slot] << 8));
            arm[2 * ((size_t)y * X + x) + 1] = v;
            // the fused kernel reads the up/down arms of output row y in row y + wy
            armc[2 * armc_index(y + wy, x, X) + 1] = v;
        }
    }
}

// Both passes in one launch: the first 2 nhx nhy CTAs run pass H, the rest
// pass V. The passes read only the grey images and write different halves of
// the arm words, so they need no order between them.
__global__ void __launch_bounds__(kSupNT) support_kernel(const __grid_constant__ SupportArgs A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    pdl_trigger();
    pdl_wait();                                   // the grey images of the previous kernel
    const int nh = A.nhx * A.nhy;
    int b = blockIdx.x;
    if (b < 2 * nh) {
        support_h(A, smem, b % A.nhx, (b / A.nhx) % A.nhy, b / nh);
    } else {
        b -= 2 * nh;
        const int nv = A.nvx * A.nvy;
        support_v(A, smem, b % A.nvx, (b / A.nvx) % A.nvy, b / nv);
    }
}

__global__ void unpack_kernel(const uint32_t *__restrict__ pix, const uint32_t *__restrict__ arm,
                              uint8_t *grey, uint8_t *census, uint32_t *arms, long n)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t p = pix[i];
    if (grey) grey[i] = (uint8_t)(p & 0xFF);
    if (census) census[i] = (uint8_t)((p >> 8) & 0x3F);
    if (arms) arms[i] = arm[i];
}

}  // namespace

cudaError_t launch_grey(const uint8_t *rgb_l, const uint8_t *rgb_r, uint8_t *g_l, uint8_t *g_r,
                        int W, int H, cudaStream_t s)
{
    long n = (long)W * H;
    long quads = (n + 3) / 4;
    dim3 grid((unsigned)((quads + 255) / 256), 2);
    bool aligned = ((reinterpret_cast<uintptr_t>(rgb_l) | reinterpret_cast<uintptr_t>(rgb_r)) & 3) == 0;
    if (aligned)
        grey_kernel<true><<<grid, 256, 0, s>>>(rgb_l, rgb_r, g_l, g_r, n);
    else
        grey_kernel<false><<<grid, 256, 0, s>>>(rgb_l, rgb_r, g_l, g_r, n);
    return cudaGetLastError();
}

cudaError_t launch_downscale(const uint8_t *g_l, const uint8_t *g_r, uint8_t *s_l, uint8_t *s_r,
                             int W, int H, cudaStream_t s)
{
    int X = W / 2, Y = H / 2;
    dim3 grid((X + 127) / 128, Y, 2);
    downscale_kernel<<<grid, 128, 0, s>>>(g_l, g_r, s_l, s_r, W, H);
    return cudaGetLastError();
}

cudaError_t launch_grey_down(const uint8_t *rgb_l, const uint8_t *rgb_r, uint8_t *gf_l, uint8_t *gf_r,
                            uint8_t *s_l, uint8_t *s_r, int W, int H, cudaStream_t s, int *launches)
{
    const int X = W / 2, Y = H / 2;
    if (X < 1 || Y < 1) return cudaErrorInvalidValue;
    const bool aligned = ((reinterpret_cast<uintptr_t>(rgb_l) | reinterpret_cast<uintptr_t>(rgb_r) |
                           reinterpret_cast<uintptr_t>(gf_l)) & 3) == 0;
    if (W % 4 != 0 || !aligned) {
        // rows not word-aligned: the two separate passes
        *launches += 2;
        cudaError_t e = launch_grey(rgb_l, rgb_r, gf_l, gf_r, W, H, s);
        return e != cudaSuccess ? e : launch_downscale(gf_l, gf_r, s_l, s_r, W, H, s);
    }
    // W a multiple of 4: a thread's group of four lies inside the row
    const int ncol = W / 4, nband = ((H + 1) / 2 + kGDB - 1) / kGDB;
    const long nthr = (long)ncol * nband;
    dim3 grid((unsigned)((nthr + kGDT - 1) / kGDT), 2);
    *launches += 1;
    return launch_dependent(grey_down_kernel, grid, dim3(kGDT), 0, s, rgb_l, rgb_r, gf_l, s_l, s_r, W, H, ncol, nband);
}

cudaError_t launch_support(const uint8_t *g_l, const uint8_t *g_r, uint32_t *pix_l, uint32_t *pix_r,
                           uint32_t *arm_l, uint32_t *arm_r, uint32_t *armc_l, uint32_t *armc_r,
                           uint32_t *key_l, uint32_t *key_r, uint32_t *err, int X, int Y, int wx, int wy,
                           int tc, cudaStream_t s)
{
    if (wx > kMaxWx || wy > kMaxWy) return cudaErrorInvalidValue;
    SupportArgs A{g_l, g_r, pix_l, pix_r, arm_l, arm_r, armc_l, armc_r, key_l, key_r, err, X, Y, wx, wy, tc,
                  (X + kHX - 1) / kHX, (Y + kHY - 1) / kHY, (X + kVX - 1) / kVX, (Y + kVY - 1) / kVY};
    const int blocks = 2 * (A.nhx * A.nhy + A.nvx * A.nvy);
    return launch_dependent(support_kernel, dim3(blocks), dim3(kSupNT),
                            (size_t)(kSupSmemH > kSupSmemV ? kSupSmemH : kSupSmemV), s, A);
}

cudaError_t launch_unpack_planes(const uint32_t *pix, const uint32_t *arm, uint8_t *grey,
                                 uint8_t *census, uint32_t *arms, int X, int Y, cudaStream_t s)
{
    long n = (long)X * Y;
    unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pix, arm, grey, census, arms, n);
    return cudaGetLastError();
}

}  // namespace stereo
