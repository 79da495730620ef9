// Fused matching cost + cross-based aggregation + winner-take-all for both
// base images: Eqs. 3-9 of the paper (Sec. III-B, III-C) in one kernel.
//
// The paper (Steps 3 and 5 of Sec. IV) writes the x-aggregated volume CA_x to
// global memory and reads it back for the y pass. Here nothing of the volume
// leaves the SM: each CTA sweeps its tile top to bottom and keeps, per
// (column, disparity), a ring of 64 running vertical prefix sums in shared
// memory.
//
// Tile: one CTA owns a strip of XS columns for each base and a slab of DS
// disparities [d0, d0+DS).
//  * Left base columns:  x in [x0, x0+XS).
//  * Right base columns: x in [x0-d0, x0-d0+XS). Shearing the right strip by
//    d0 makes both bases read one row of left-base costs: by Eq. 6,
//    C^R(x, y, d) = C^L(x+d, y, d), and for d in the slab the right windows
//    land inside [x0-wx, x0+XS+DS-1+wx), next to the left windows.
//
// Per input row y and disparity d (phase A, one warp per (row, d)):
//    S[i] = sum_{j<i} C^L(x0 - wx + j, y, d)     (row prefix, exact uint32)
// where C^L is P when the match pixel x-d or the pixel itself is outside
// the image. Each lane sums four consecutive costs, then a warp scan adds the
// lanes' totals.
// Per pixel (phase B, one thread per (base, column, 3 disparities)):
//    CA_x = S[hi] - S[lo] over the pixel's own left/right arms   (Eq. 7)
//    V(y+1) = V(y) + CA_x   -> ring slot (y+1) mod 64
//    CA(yo) = V(yo + down + 1) - V(yo - up), yo = y - wy         (Eq. 8)
//    key = min over d of (CA << 8 | d)                            (Eq. 9)
// The min over slabs is an atomicMin on a 32-bit key per pixel and base. The
// packed key keeps the smallest d among equal costs, the tie rule of Step 5.
// All sums are modular uint32: differences are exact because every window sum
// is below 2^24 (checked on the host).
#include "internal.cuh"

namespace stereo {
namespace {

constexpr int XS = 64;              // columns per base per CTA
constexpr int DS = 6;               // disparities per CTA
constexpr int NG = 2;               // disparity groups per (base, column)
constexpr int DPT = DS / NG;        // disparities per thread
constexpr int RB = 4;               // rows per phase A / phase B round
constexpr int NT = 2 * XS * NG;     // 256 threads
constexpr int NW = NT / 32;
constexpr int KE = 4;               // prefix entries per lane in phase A
constexpr int SWP = 176;            // S row pitch in words (== 16 mod 32)
constexpr int SX_OFF = 3;           // S[i] at word SX_OFF + i: S[1 + 4 lane] is 16-byte aligned
constexpr int LUT_N = 256 * 8;
constexpr int RING_J = NG * XS;                 // words between disparities of a ring row
constexpr int RING_SLOT = DPT * RING_J;         // words per ring slot
constexpr int RING_BASE = kRing * RING_SLOT;    // words per base
constexpr int SMEM_WORDS = LUT_N + RB * DS * SWP + 2 * RING_BASE;

static_assert(32 * KE + SX_OFF + 1 <= SWP, "S row too short");
static_assert(SWP % 32 == 16, "S pitch chosen so the two disparity groups use different banks");
static_assert(NW == 8 && XS == 64, "warp -> (base, 16-column group) mapping assumes 8 warps");

__global__ void __launch_bounds__(NT, 1) costagg_wta_kernel(const CostAggArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *lut = smem;
    uint32_t *sx = lut + LUT_N;
    uint32_t *ring = sx + RB * DS * SWP;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int X = a.X, Y = a.Y, D = a.D, wx = a.wx, wy = a.wy;
    const int x0 = blockIdx.x * XS;
    const int d0 = blockIdx.y * DS;
    const uint32_t P = a.P;

    for (int i = tid; i < LUT_N; i += NT) lut[i] = a.lut[i];

    // Phase B identity: warps 0-3 left base, 4-7 right base; a warp covers 16
    // columns and both disparity groups (lane bit 4).
    const int b = warp >> 2;
    const int xl = ((warp & 3) << 4) + (lane & 15);
    const int g = lane >> 4;
    const int col = b == 0 ? x0 + xl : x0 - d0 + xl;
    const bool valid = col >= 0 && col < X;
    const uint32_t *arm = b ? a.arm_r : a.arm_l;
    uint32_t *key = b ? a.key_r : a.key_l;
    // The two groups of a warp sit XS words apart; xor-ing bit 4 of the column
    // for group 1 puts the 32 lanes of a ring access in 32 different banks.
    uint32_t *myring = ring + b * RING_BASE + g * XS + (xl ^ (g << 4));

    uint32_t V[DPT];
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        V[j] = 0;
        myring[j * RING_J] = 0;          // slot 0 holds V(0) = 0
    }
    __syncthreads();

    const int NE = XS + DS - 1 + 2 * wx;   // S[0..NE]

    for (int yb = 0; yb < Y + wy; yb += RB) {
        // ---------------- phase A: cost + row prefix for RB rows x DS disparities
        for (int u = warp; u < RB * DS; u += NW) {
            const int r = u / DS, dd = u - r * DS;
            const int y = yb + r, d = d0 + dd;
            if (y >= Y || d >= D) continue;                  // warp-uniform
            const uint32_t *pl = a.pix_l + (size_t)y * X;
            const uint32_t *pr = a.pix_r + (size_t)y * X;
            uint32_t c[KE];
            uint32_t run = 0;
#pragma unroll
            for (int k = 0; k < KE; ++k) {
                const int i = lane * KE + k;
                const int xL = x0 - wx + i;
                uint32_t v = 0;
                if (i < NE) {
                    if (xL >= d && xL < X) {
                        const uint32_t p = __ldg(pl + xL), q = __ldg(pr + xL - d);
                        const int ad = abs((int)(p & 0xFF) - (int)(q & 0xFF));
                        const int hd = __popc((p ^ q) >> 8);
                        v = lut[ad * 8 + hd];
                    } else {
                        v = P;
                    }
                }
                run += v;
                c[k] = run;
            }
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t excl = incl - run;
            uint32_t *row = sx + (r * DS + dd) * SWP + SX_OFF;
            *reinterpret_cast<uint4 *>(row + 1 + lane * KE) =
                make_uint4(excl + c[0], excl + c[1], excl + c[2], excl + c[3]);
            if (lane == 0) row[0] = 0;
        }
        __syncthreads();

        // ---------------- phase B: arm differences, vertical ring, WTA
#pragma unroll 1
        for (int r = 0; r < RB; ++r) {
            const int y = yb + r;
            if (y < Y) {
                const uint32_t am = valid ? __ldg(arm + (size_t)y * X + col) : 0u;
                const int hm = am & 0xFF, hp = (am >> 8) & 0xFF;
                const int slot = (y + 1) & (kRing - 1);
#pragma unroll
                for (int j = 0; j < DPT; ++j) {
                    const int dd = g * DPT + j;
                    const int base = xl + (b ? dd : 0) + wx;
                    const uint32_t *row = sx + (r * DS + dd) * SWP + SX_OFF;
                    V[j] += row[base + hp + 1] - row[base - hm];
                    myring[slot * RING_SLOT + j * RING_J] = V[j];
                }
            }
            const int yo = y - wy;
            if (yo >= 0 && yo < Y) {
                const uint32_t am = valid ? __ldg(arm + (size_t)yo * X + col) : 0u;
                const int vm = (am >> 16) & 0xFF, vp = am >> 24;
                const int shi = (yo + vp + 1) & (kRing - 1);
                const int slo = (yo - vm) & (kRing - 1);
                uint32_t best = 0xFFFFFFFFu;
#pragma unroll
                for (int j = 0; j < DPT; ++j) {
                    const int d = d0 + g * DPT + j;
                    const uint32_t ca = myring[shi * RING_SLOT + j * RING_J] - myring[slo * RING_SLOT + j * RING_J];
                    if (d < D) best = min(best, (ca << 8) | (uint32_t)d);
                }
                best = min(best, __shfl_xor_sync(0xffffffffu, best, 16));
                if (g == 0 && valid) atomicMin(key + (size_t)yo * X + col, best);
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t costagg_smem_bytes(int wx)
{
    if (wx < 0 || XS + DS - 1 + 2 * wx > 32 * KE) return 0;
    return (size_t)SMEM_WORDS * 4;
}

cudaError_t costagg_setup()
{
    return cudaFuncSetAttribute(costagg_wta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_WORDS * 4);
}

cudaError_t launch_costagg(const CostAggArgs &a, cudaStream_t s)
{
    size_t smem = costagg_smem_bytes(a.wx);
    if (smem == 0 || a.wy > kMaxWy || a.wy < 0) return cudaErrorInvalidValue;
    const int nslab = (a.D + DS - 1) / DS;
    const int dlast = (nslab - 1) * DS;
    const int nstrip = (a.X + dlast + XS - 1) / XS;
    dim3 grid(nstrip, nslab);
    costagg_wta_kernel<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace stereo
