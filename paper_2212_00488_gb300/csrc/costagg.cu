// Fused matching cost + cross-based aggregation + winner-take-all for both
// base images: Eqs. 3-9 of the paper (Sec. III-B, III-C) in one kernel.
//
// The paper (Steps 3 and 5 of Sec. IV) writes the x-aggregated volume CA_x to
// global memory and reads it back for the y pass. Here nothing of the volume
// leaves the SM: each CTA sweeps its tile top to bottom and keeps, per
// (column, disparity, base), a ring of 64 running vertical prefix sums in
// shared memory.
//
// Tile: one CTA owns a strip of XS columns for each base and a slab of DS
// disparities [d0, d0+DS).
//  * Left base columns:  x in [x0, x0+XS).
//  * Right base columns: x in [x0-d0, x0-d0+XS). Shearing the right strip by
//    d0 makes both bases read one row of left-base costs: by Eq. 6,
//    C^R(x, y, d) = C^L(x+d, y, d), and for d in the slab the right windows
//    land inside [x0-wx, x0+XS+DS-1+wx), next to the left windows.
//
// Warp roles (the row buffers between them form a ring of RS slots; rows
// 4k..4k+3 share one full and one empty mbarrier):
//  * Producer warp p (NPW of them) fills rows y = p, p + NPW, ...: for each
//    disparity d = d0 + q of the slab, the exclusive row prefix
//      S_q[i] = sum_{j<i} C^L(x0 - wx + j, y, d)                  (Eq. 7)
//    with C^L = P when the pixel or its match x - d is outside the image.
//    Each lane sums KE consecutive costs (one table lookup each: the AD and
//    census terms of Eqs. 3-5 combined), a warp scan adds the lanes' totals.
//    Prefixes are exact modulo 2^16 or 2^32 (16-bit only when every
//    horizontal window sum is below 2^16, checked on the host).
//  * Consumer thread (base, column) holds the slab's DS = 4 disparities and
//    takes four rows per step:
//      CA_x = S_q[hi] - S_q[lo] over the pixel's own left/right arms  (Eq. 7)
//      V(y+1) = V(y) + CA_x  -> ring slot y mod 64
//      CA(yo) = V(yo + down + 1) - V(yo - up), yo = y - wy          (Eq. 8)
//      key = min over d of (CA << 8 | d)                             (Eq. 9)
//    The minimum over slabs is one atomicMin per pixel and base. The packed
//    key keeps the smallest d among equal costs, the tie rule of Step 5.
// Vertical sums are modular uint32 and kept multiplied by 256 (V << 8): a
// difference of two ring entries is then CA << 8 exactly, because every
// window sum is below 2^24 (checked on the host), and a key is one add of d.
// A column's arm words of four rows arrive in one 16-byte load (armc_index).
//
// Every wait on an mbarrier is bounded: after a.wait_limit polls the thread
// sets a.err and returns, so a broken hand-off ends the kernel with an error
// status instead of hanging the GPU.
#include "internal.cuh"

#include <type_traits>

namespace stereo {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}

// One poll of the phase with the given parity. A thread whose phase is not
// complete is suspended until the phase completes or at most kSuspendNs have
// passed, so waiting warps leave the issue slots to the warps doing the work.
constexpr uint32_t kSuspendNs = 1000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `bar` with the given parity to complete,
// warp-uniform: the warp goes on only if every lane saw the phase complete.
// After `limit` polls (each suspends at most kSuspendNs) the error word is set
// and false is returned to every lane.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, uint32_t limit, uint32_t *err)
{
    bool ok = false;
    for (uint32_t it = 0; !ok && it < limit; ++it) ok = mbar_try_wait(bar, parity);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(err, 1u);
    return ok;
}

// Combined cost table: entry (h, ad) = AD(ad) + MC(h) at h * kLutPitch + ad
// (16-bit entries; Hamming distances 0..6). A row pitch of 136 words moves
// the rows of successive h by 8 banks, so lanes with small ad and small h
// read distinct banks.
constexpr int kLutRows = 7;
constexpr int kLutPitch = 272;

template <int XS_, int DS_, int KE_, int RS_, bool S16_, int DPT_, int NPW_>
struct Tile {
    static constexpr int XS = XS_;            // columns per base
    static constexpr int DS = DS_;            // disparities per CTA
    static constexpr int KE = KE_;            // prefix entries per producer lane (odd)
    static constexpr int RS = RS_;            // row slots between producers and consumers
    static constexpr bool S16 = S16_;         // row prefixes kept mod 2^16 (window sums < 2^16)
    static constexpr int DPT = DPT_;          // disparities per consumer thread
    using SType = typename std::conditional<S16_, uint16_t, uint32_t>::type;
    static constexpr int G = DS / DPT;        // consumer threads per column (adjacent lanes)
    static constexpr int LPX = 32 / G;        // columns per consumer warp
    static constexpr int NCT = 2 * XS * G;    // consumer threads with a column
    static constexpr int NCTP = (NCT + 31) / 32 * 32;   // consumer threads, whole warps
    static constexpr int NPW = NPW_;          // producer warps; warp p fills rows y = p (mod NPW)
    static constexpr int NP = 32 * NPW;
    static constexpr int NT = NCTP + NP;
    static constexpr int NE = 32 * KE;        // S[0..NE]
    // S row pitch in elements: the G groups of a consumer warp read rows that
    // start LPX words apart modulo the 32 banks (with one group any pitch does)
    static constexpr int SWP = NE + (G == 1 ? 4 : S16 ? 2 * LPX : LPX);
    static constexpr int NB = RS / 4;         // row quads share a full and an empty barrier
    static constexpr int B_BAR = 2 * NB * 8;
    static constexpr int B_RING = kRing * NCT * DPT * 4;
    // 16-bit prefixes: the prefixes of disparities 2j and 2j+1 at one column
    // share a 32-bit word (pair plane j, SWP words per plane); 32-bit
    // prefixes: one plane per disparity, SWP words each. Same bytes.
    static constexpr int B_SX = RS * DS * SWP * (int)sizeof(SType);
    static constexpr int B_LUT = kLutRows * kLutPitch * 2;
    static constexpr int BYTES = B_BAR + B_RING + B_SX + B_LUT;
    static_assert(DS % DPT == 0 && 32 % G == 0, "the threads of a column sit in adjacent lanes of one warp");
    static_assert(DPT == 4, "ring entries are 16 bytes");
    static_assert(!S16 || (DS == 4 && G == 1), "pair planes hold the slab's four disparities");
    static_assert(KE % 2 == 1, "odd KE keeps the producer lanes' strided stores in distinct banks");
    static_assert(NT <= 1024, "");
    static_assert(RS == NPW, "producer warp p owns row slot p");
    static_assert(RS % 4 == 0, "slots are handed over in row quads");
    static_assert(BYTES <= 232448, "tile exceeds shared memory");
};

template <int N> struct VecOf;
template <> struct VecOf<4> { using type = uint4; };

template <int N>
__device__ __forceinline__ uint32_t &vget(typename VecOf<N>::type &v, int k);
template <>
__device__ __forceinline__ uint32_t &vget<4>(uint4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One tile (x-strip from x0, disparity slab from d0) of one frame. `reuse`
// is set when this CTA already ran a tile: its barriers are invalidated before
// they are initialised again and the cost table is already in place.
template <class T>
__device__ __forceinline__ void costagg_tile(const CostAggArgs &a, const int x0, const int d0,
                                             unsigned char *smem, const bool reuse)
{
    using SType = typename T::SType;
    using Vec = typename VecOf<T::DPT>::type;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + T::NB;
    Vec *ring = reinterpret_cast<Vec *>(smem + T::B_BAR);                     // [64][NCT]
    SType *sx = reinterpret_cast<SType *>(smem + T::B_BAR + T::B_RING);       // [RS][DS][SWP] (32-bit)
    uint32_t *sxw = reinterpret_cast<uint32_t *>(sx);                           // [RS][2][SWP] (16-bit pairs)
    uint16_t *lut = reinterpret_cast<uint16_t *>(smem + T::B_BAR + T::B_RING + T::B_SX);  // [7][kLutPitch]

    const int t = threadIdx.x, lane = t & 31;
    const int X = a.X, Y = a.Y, D = a.D, wx = a.wx, wy = a.wy;
    const uint32_t limit = a.wait_limit;

    // combined cost table: AD(|grey difference|) + MC(Hamming)
    if (!reuse)
        for (int i = t; i < kLutRows * kLutPitch; i += T::NT) {
            const int h = i / kLutPitch, ad = i - h * kLutPitch;
            lut[i] = ad < 256 ? (uint16_t)(a.lut_ad[ad] + a.lut_mc[h]) : (uint16_t)0;
        }
    if (t == 0) {
        for (int s = 0; s < T::NB; ++s) {
            if (reuse) {
                mbar_inval(&full[s]);
                mbar_inval(&empty[s]);
            }
            mbar_init(&full[s], 128);               // the four producing warps of a row quad
            mbar_init(&empty[s], T::NCTP);          // every consumer thread
        }
    }
    if (!reuse) pdl_wait();                       // the support words and keys of the previous kernel
    __syncthreads();

    if (t >= T::NCTP) {
        // ======================= producers: warp pw fills rows pw, pw + NPW, ... in slot pw
        const int pw = (t - T::NCTP) >> 5;
        const uint32_t P = a.P;
        const int xb = x0 - wx + lane * T::KE;      // x of this lane's first entry
        // per-lane constants: clamped load offsets and, per (entry, disparity),
        // whether the pixel and its match lie in the image
        int offl[T::KE], offr[T::KE + T::DS - 1];
        using Mask = typename std::conditional<(T::KE * T::DS > 32), uint64_t, uint32_t>::type;
        Mask inimg = 0;
#pragma unroll
        for (int k = 0; k < T::KE; ++k) offl[k] = min(max(xb + k, 0), X - 1);
#pragma unroll
        for (int k = 0; k < T::KE + T::DS - 1; ++k) offr[k] = min(max(xb + k - d0 - (T::DS - 1), 0), X - 1);
#pragma unroll
        for (int k = 0; k < T::KE; ++k)
#pragma unroll
            for (int q = 0; q < T::DS; ++q)
                if (xb + k >= d0 + q && xb + k < X) inimg |= (Mask)1 << (k * T::DS + q);
        const bool all_in = __all_sync(0xffffffffu, inimg == (Mask)(~(Mask)0 >> (8 * sizeof(Mask) - T::KE * T::DS)));
        // pixels of one row: the lane's KE entries and their KE + DS - 1 matches
        uint32_t pv0[T::KE], qv0[T::KE + T::DS - 1];
        auto load = [&](int y, uint32_t (&pv)[T::KE], uint32_t (&qv)[T::KE + T::DS - 1]) {
            if (y >= Y) return;
            const uint32_t *pl = a.pix_l + (size_t)y * X;
            const uint32_t *pr = a.pix_r + (size_t)y * X;
            if (all_in) {
                // every entry and match lies in the image: one base per row,
                // the entries at fixed offsets from it
                const uint32_t *bl = pl + xb, *br = pr + (xb - d0 - (T::DS - 1));
#pragma unroll
                for (int k = 0; k < T::KE; ++k) pv[k] = __ldg(bl + k);
#pragma unroll
                for (int k = 0; k < T::KE + T::DS - 1; ++k) qv[k] = __ldg(br + k);
            } else {
#pragma unroll
                for (int k = 0; k < T::KE; ++k) pv[k] = __ldg(pl + offl[k]);
#pragma unroll
                for (int k = 0; k < T::KE + T::DS - 1; ++k) qv[k] = __ldg(pr + offr[k]);
            }
        };
        // The next row's pixels are loaded into the same registers as soon
        // as this row's costs are formed, and the wait for a free slot comes
        // after the scan, so load latency and hand-off overlap the work.
        load(pw, pv0, qv0);
        // matching cost of entry k at disparity d0 + q (its match is qv index
        // k + DS-1 - q): one table lookup for the AD and census terms, or P
        // outside the image (only warps that touch a border test it)
        auto cost = [&](auto border, int k, int q) -> uint32_t {
            constexpr bool kBorder = decltype(border)::value;
            const uint32_t pk = pv0[k], qk = qv0[k + T::DS - 1 - q];
            const uint32_t ad = __vabsdiffu4(pk, qk) & 0xFFu;     // |grey difference| from the low bytes
            uint32_t v = lut[__popc((pk ^ qk) & 0x3F00u) * kLutPitch + ad];
            if (kBorder) v = (inimg >> (k * T::DS + q)) & 1u ? v : P;
            return v;
        };
        uint32_t ph = 1;                            // parity of the empty phase to wait for
        const int s = pw;                           // this warp's row slot
        for (int y = pw; y < Y; y += T::NPW, ph ^= 1u) {
            if constexpr (T::S16) {
                // 16-bit prefixes: the costs of disparities 2j and 2j+1 travel
                // as the halves of one word (pair plane j). A lane's running
                // sums stay below 2^16 (KE P < 2^16, checked on the host), so
                // plain adds do; across lanes the halves add modulo 2^16 each.
                uint32_t c2[2][T::KE], run2[2] = {0u, 0u};
                auto form = [&](auto border) {
#pragma unroll
                    for (int k = 0; k < T::KE; ++k)
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            run2[j] += __byte_perm(cost(border, k, 2 * j), cost(border, k, 2 * j + 1), 0x5410);
                            c2[j][k] = run2[j];
                        }
                };
                if (all_in)
                    form(std::false_type{});
                else
                    form(std::true_type{});
                load(y + T::NPW, pv0, qv0);
                uint32_t incl2[2] = {run2[0], run2[1]};
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t u = __shfl_up_sync(0xffffffffu, incl2[j], o);
                        if (lane >= o) incl2[j] = __vadd2(incl2[j], u);
                    }
                }
                if (y >= T::RS && !mbar_wait_warp(&empty[s >> 2], ph, limit, a.err)) return;
                // lanes write words KE apart (KE odd): no bank conflicts
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t e2 = __vsub2(incl2[j], run2[j]);   // exclusive prefix of the lane's first entry
                    uint32_t *row = sxw + (s * 2 + j) * T::SWP;
#pragma unroll
                    for (int k = 0; k < T::KE; ++k) row[1 + lane * T::KE + k] = __vadd2(e2, c2[j][k]);
                    if (lane == 0) row[0] = 0;
                }
            } else {
                uint32_t c[T::DS][T::KE];
                uint32_t run[T::DS];
                auto form = [&](auto border) {
#pragma unroll
                    for (int q = 0; q < T::DS; ++q) run[q] = 0;
#pragma unroll
                    for (int k = 0; k < T::KE; ++k)
#pragma unroll
                        for (int q = 0; q < T::DS; ++q) {
                            run[q] += cost(border, k, q);
                            c[q][k] = run[q];
                        }
                };
                if (all_in)
                    form(std::false_type{});
                else
                    form(std::true_type{});
                load(y + T::NPW, pv0, qv0);
                uint32_t incl[T::DS];
#pragma unroll
                for (int q = 0; q < T::DS; ++q) incl[q] = run[q];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                    for (int q = 0; q < T::DS; ++q) {
                        const uint32_t u = __shfl_up_sync(0xffffffffu, incl[q], o);
                        if (lane >= o) incl[q] += u;
                    }
                }
                if (y >= T::RS && !mbar_wait_warp(&empty[s >> 2], ph, limit, a.err)) return;
#pragma unroll
                for (int q = 0; q < T::DS; ++q) {
                    const uint32_t excl = incl[q] - run[q];
                    SType *row = sx + (s * T::DS + q) * T::SWP;
#pragma unroll
                    for (int k = 0; k < T::KE; ++k) row[1 + lane * T::KE + k] = (SType)(excl + c[q][k]);
                    if (lane == 0) row[0] = 0;
                }
            }
            mbar_arrive(&full[s >> 2]);
            if (y + 1 == Y)                               // the quad's rows that do not exist
                for (int k = y & 3; k < 3; ++k) mbar_arrive(&full[s >> 2]);
        }
        return;
    }

    // =========================== consumers: thread (base, column, DPT disparities)
    // thread t: group g = t mod G, column index t / G over both bases (a warp
    // may hold columns of both bases; the G threads of a column never straddle
    // warps since G divides 32)
    const int g = t & (T::G - 1);                 // disparity group of this thread
    const int ci = t / T::G;
    // threads past the last column only keep the hand-off going
    const bool active = T::NCT == T::NCTP || t < T::NCT;
    const int b = ci >= T::XS;
    const int x = active ? ci - b * T::XS : T::XS - 1;
    const int col = b ? x0 - d0 + x : x0 + x;
    const bool valid = active && col >= 0 && col < X;
    const int colc = min(max(col, 0), X - 1);
    const int dg = d0 + g * T::DPT;               // first disparity of the group
    uint32_t *key = (b ? a.key_r : a.key_l) + colc;
    // combined arm words, four rows per 16-byte quad (armc_index): row r holds
    // the left/right arms of row r (low half) and the up/down arms of row
    // r - wy (high half)
    const uint4 *armq = reinterpret_cast<const uint4 *>(b ? a.armc_r : a.armc_l) + colc;
    // ring entries of this thread (an idle thread reads the last column's
    // entries and never writes)
    Vec *myring = ring + (active ? t : T::NCT - 1);
    // S element of this pixel's own column for the group's first disparity
    const SType *srow0 = sx + (g * T::DPT) * T::SWP + x + wx + (b ? g * T::DPT : 0);
    const int rows = Y + wy;                      // row steps: inputs 0..Y-1, outputs lag by wy
    const int nquad = (rows + 3) >> 2;            // arm-word quads

    if (active) {
        Vec z;
#pragma unroll
        for (int k = 0; k < T::DPT; ++k) vget<T::DPT>(z, k) = 0;
        myring[(kRing - 1) * T::NCT] = z;         // V(0) = 0 (V(r) sits in slot (r - 1) mod 64)
    }
    uint32_t V[T::DPT];
#pragma unroll
    for (int k = 0; k < T::DPT; ++k) V[k] = 0;

    // pair plane 0 of slot 0 at this pixel's own column (16-bit prefixes)
    const uint32_t *wrow0 = sxw + x + wx;
    // x-window sums of one input row for this thread's disparities, times 256
    // (modulo 2^32). With 16-bit prefixes a warp of left-base columns (kLeft)
    // reads both disparities of a pair plane with one 32-bit load; right-base
    // columns read disparity k at column + k, so each half on its own. A byte
    // permutation takes a 16-bit difference and places it at bits 8..23.
    auto hsum = [&](auto left, int slot, uint32_t am, uint32_t (&cax)[T::DPT]) {
        [[maybe_unused]] constexpr bool kLeft = decltype(left)::value;
        const int hi = ((am >> 8) & 0xFF) + 1, lo = am & 0xFF;
        if constexpr (T::S16) {
            const uint32_t *w = wrow0 + slot * (2 * T::SWP);
            if constexpr (kLeft) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    // both disparities of the pair at once, each half modulo 2^16
                    const uint32_t dd = __vsub2(w[j * T::SWP + hi], w[j * T::SWP - lo]);
                    cax[2 * j] = __byte_perm(dd, 0u, 0x4104);
                    cax[2 * j + 1] = __byte_perm(dd, 0u, 0x4324);
                }
            } else {
#pragma unroll
                for (int k = 0; k < T::DPT; ++k) {
                    const uint16_t *hk = reinterpret_cast<const uint16_t *>(w + (k >> 1) * T::SWP + (b ? k : 0)) + (k & 1);
                    cax[k] = __byte_perm((uint32_t)hk[2 * hi] - (uint32_t)hk[-2 * lo], 0u, 0x4104);
                }
            }
        } else {
            const SType *r0 = srow0 + slot * (T::DS * T::SWP);
#pragma unroll
            for (int k = 0; k < T::DPT; ++k) {
                const SType *rk = r0 + k * (T::SWP + (b ? 1 : 0));
                cax[k] = ((uint32_t)rk[hi] - (uint32_t)rk[-lo]) << 8;
            }
        }
    };
    // V(y + 1) into ring slot y mod 64; the four rows of a step (y a
    // multiple of 4) land in consecutive slots of one step base
    auto push = [&](Vec *step_base, int j, const uint32_t (&cax)[T::DPT]) {
        Vec w;
#pragma unroll
        for (int k = 0; k < T::DPT; ++k) {
            V[k] += cax[k];
            vget<T::DPT>(w, k) = V[k];
        }
        if (active) step_base[j * T::NCT] = w;
    };
    // Four rows per step, one wait per step. While all four rows are inputs
    // the step has no branch but the wait, so the loads and arithmetic of
    // the rows interleave; idle threads and rows without an output do the
    // same work and drop it. Arm words are fetched a step ahead. Slabs that
    // lie wholly below D run without the per-disparity range test.
    auto sweep = [&](auto part, auto left) {
        constexpr bool kPart = decltype(part)::value;
        // packed WTA key of output row yo over this thread's disparities
        auto vkey = [&](int yo, uint32_t am) -> uint32_t {
            const int up = (am >> 16) & 0xFF, down = am >> 24;
            Vec vh = myring[((yo + down) & (kRing - 1)) * T::NCT];      // V(yo + down + 1)
            Vec vl = myring[((yo - up - 1) & (kRing - 1)) * T::NCT];    // V(yo - up)
            uint32_t best = 0xFFFFFFFFu;
#pragma unroll
            for (int k = 0; k < T::DPT; ++k) {
                // (V(hi) - V(lo)) << 8 is CA << 8 exactly: the key (CA << 8 | d) is one add
                const uint32_t kk = vget<T::DPT>(vh, k) - vget<T::DPT>(vl, k) + (uint32_t)(dg + k);
                best = (!kPart || dg + k < D) ? min(best, kk) : best;
            }
            return best;
        };
        constexpr int R = 4;                      // rows per step: one arm-word quad
        uint4 am = __ldg(armq);
        auto atomics = [&](auto inputs, int y, uint32_t (&kk)[R]) {
            constexpr bool kInputs = decltype(inputs)::value;   // rows y .. y+3 all exist
            // the G threads of a column (adjacent lanes) combine their
            // disparity groups' minima; one atomic per column and row
            if constexpr (T::G > 1) {
#pragma unroll
                for (int j = 0; j < R; ++j)
#pragma unroll
                    for (int o = 1; o < T::G; o <<= 1) kk[j] = min(kk[j], __shfl_xor_sync(0xffffffffu, kk[j], o));
            }
            if (g == 0 && valid) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if (y + j - wy >= 0 && (kInputs || y + j < rows)) atomicMin(key + (y + j - wy) * X, kk[j]);
            }
        };
        int y = 0;
        int ys = 0;                               // slot of row y (rows y + j take ys + j)
        uint32_t ph = 0;                          // parity of the full phase of those slots
        auto next_slots = [&]() {
            ys += R;
            if (ys == T::RS) {
                ys = 0;
                ph ^= 1u;
            }
        };
        // steps whose four rows are all inputs: no branch but the wait
        for (; y + R - 1 < Y; y += R) {
            const uint4 an = __ldg(armq + min((y >> 2) + 1, nquad - 1) * X);
            uint32_t c[R][T::DPT], kk[R];
            Vec *const sb = myring + (y & (kRing - 1)) * T::NCT;
            if (!mbar_wait_warp(&full[ys >> 2], ph, limit, a.err)) return;
#pragma unroll
            for (int j = 0; j < R; ++j) hsum(left, ys + j, vget<4>(am, j), c[j]);
            mbar_arrive(&empty[ys >> 2]);
#pragma unroll
            // output row r - wy reads V down to slot r - 2wy, which shares
            // its ring slot with r + 2 when wy = 31, so each row's key is
            // taken before the next row is pushed
            for (int j = 0; j < R; ++j) {
                push(sb, j, c[j]);
                kk[j] = vkey(y + j - wy, vget<4>(am, j));
            }
            atomics(std::true_type{}, y, kk);
            am = an;
            next_slots();
        }
        // the last input rows and the output rows that lag them
        for (; y < rows; y += R) {
            const uint4 an = __ldg(armq + min((y >> 2) + 1, nquad - 1) * X);
            uint32_t c[R][T::DPT], kk[R];
            Vec *const sb = myring + (y & (kRing - 1)) * T::NCT;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int r = y + j;
                if (r < Y) {
                    if (j == 0 && !mbar_wait_warp(&full[ys >> 2], ph, limit, a.err))
                        return;
                    hsum(left, ys + j, vget<4>(am, j), c[j]);
                    if (j == R - 1 || r + 1 == Y) mbar_arrive(&empty[ys >> 2]);
                    push(sb, j, c[j]);
                }
                kk[j] = vkey(r - wy, vget<4>(am, j));
            }
            atomics(std::false_type{}, y, kk);
            am = an;
            next_slots();
        }
    };
    // warps whose columns are all of the left base take the paired loads
    const bool left_warp = __all_sync(0xffffffffu, b == 0);
    auto run = [&](auto part) {
        if constexpr (T::S16) {
            if (left_warp)
                sweep(part, std::true_type{});
            else
                sweep(part, std::false_type{});
        } else {
            sweep(part, std::false_type{});
        }
    };
    if (d0 + T::DS <= D)
        run(std::false_type{});
    else
        run(std::true_type{});
}

// Tiles of a frame, slab by slab. Slab s (first disparity d0 = s DS) needs
// strips x0 = 0, XS, ... until both bases are covered: the left base reads
// columns [x0, x0 + XS), the right base [x0 - d0, x0 - d0 + XS), so
// ceil((X + d0) / XS) strips; low slabs need fewer than high ones.
template <class T>
__host__ __device__ __forceinline__ int slab_strips(const CostAggArgs &a, int slab)
{
    return (a.X + slab * T::DS + T::XS - 1) / T::XS;
}

template <class T>
__host__ __device__ __forceinline__ int tiles_of(const CostAggArgs &a)
{
    int n = 0;
    for (int s = 0; s * T::DS < a.D; ++s) n += slab_strips<T>(a, s);
    return n;
}

template <class T>
__device__ __forceinline__ void tile_at(const CostAggArgs &a, int tile, int &x0, int &d0)
{
    int s = 0;
    for (int n = slab_strips<T>(a, 0); tile >= n; n = slab_strips<T>(a, s)) {
        tile -= n;
        ++s;
    }
    x0 = tile * T::XS;
    d0 = s * T::DS;
}

template <class T>
__global__ void __launch_bounds__(T::NT, 1) costagg_wta_kernel(const CostAggArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_trigger();
    int x0, d0;
    tile_at<T>(a, blockIdx.x, x0, d0);
    costagg_tile<T>(a, x0, d0, smem, false);
}

// Persistent form for a batch of frames: one CTA per SM takes tiles (job,
// strip, slab) from a global counter until none is left. Jobs come largest
// first, so the long sweeps start early and the short ones fill the tail.
template <class T>
__global__ void __launch_bounds__(T::NT, 1) costagg_batch_kernel(const __grid_constant__ BatchArgs b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_tile;
    pdl_trigger();
    bool reuse = false;
    for (;;) {
        if (threadIdx.x == 0) {
            // stop taking tiles once a bounded wait has given up anywhere
            const bool failed = *(volatile uint32_t *)b.job[0].err != 0u;
            s_tile = failed ? b.total_tiles : (int)atomicAdd(b.counter, 1u);
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= b.total_tiles) return;
        int j = 0;
        while (j + 1 < b.njobs && tile >= b.tile_start[j + 1]) ++j;
        int x0, d0;
        tile_at<T>(b.job[j], tile - b.tile_start[j], x0, d0);
        costagg_tile<T>(b.job[j], x0, d0, smem, reuse);
        reuse = true;
        __syncthreads();
    }
}

// Tile shapes (XS x DS, KE, RS, 16-bit prefixes, DPT, producer warps). One
// CTA per SM; the ring of 64 prefix rows per (column, disparity, base)
// dominates shared memory. Every shape gives the same keys.
using T0 = Tile<104, 4, 5, 8, true, 4, 8>;    // wx <= 26, window sums < 2^16
using T1 = Tile<104, 4, 7, 8, true, 4, 8>;    // wx <= 58, window sums < 2^16
using T2 = Tile<104, 4, 5, 4, false, 4, 4>;   // wx <= 26, 32-bit prefixes
using T3 = Tile<104, 4, 7, 4, false, 4, 4>;   // wx <= 58, 32-bit prefixes
using T4 = Tile<64, 4, 5, 8, true, 4, 8>;     // narrow frames, window sums < 2^16
// 100 columns leave room for 12 producer warps and row slots (19 warps per
// SM); at 718 columns every slab of a 145-disparity frame takes 8 strips,
// 152 CTAs
using T5 = Tile<100, 4, 5, 12, true, 4, 12>;
// slabs of 8 disparities: two threads per column, 32-bit prefixes (the
// batch autotuner's deeper slab)
using T6 = Tile<48, 8, 5, 4, false, 4, 4>;
// wide horizontal windows (Table I: W_x up to 141 per side), wx <= 174,
// 32-bit prefixes; 64 columns leave room for 8 producer warps and row slots
using T7 = Tile<64, 4, 13, 8, false, 4, 8>;
// wx up to 66 (Table I's W_x = 61) with 32-bit prefixes: 7 prefix entries
// per producer lane leave room for 8 producer warps and row slots
using T8 = Tile<88, 4, 7, 8, false, 4, 8>;

template <class T> struct Tag { using type = T; };

// Calls f(Tag<T>) for the tile shape with the given id; false for an unknown id.
template <class F>
bool with_tile(int id, F &&f)
{
    switch (id) {
    case 0: f(Tag<T0>{}); return true;
    case 1: f(Tag<T1>{}); return true;
    case 2: f(Tag<T2>{}); return true;
    case 3: f(Tag<T3>{}); return true;
    case 4: f(Tag<T4>{}); return true;
    case 5: f(Tag<T5>{}); return true;
    case 6: f(Tag<T6>{}); return true;
    case 7: f(Tag<T7>{}); return true;
    case 8: f(Tag<T8>{}); return true;
    default: return false;
    }
}
static_assert(kNumTiles == 9, "tile ids 0..8");

template <class T>
bool fits(const CostAggArgs &a)
{
    if (T::XS + T::DS - 1 + 2 * a.wx > T::NE) return false;
    // 16-bit prefixes need every horizontal window sum, and every producer
    // lane's sum of KE costs, below 2^16
    return !T::S16 || (uint64_t)max(2 * a.wx + 1, T::KE) * a.P < 65536u;
}


template <class T>
cudaError_t setup_one()
{
    cudaError_t e = cudaFuncSetAttribute(costagg_wta_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         T::BYTES);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(costagg_batch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, T::BYTES);
}

template <class T>
cudaError_t launch_batch_one(BatchArgs &b, int nsm, cudaStream_t s)
{
    b.total_tiles = 0;
    for (int j = 0; j < b.njobs; ++j) {
        if (!fits<T>(b.job[j])) return cudaErrorInvalidValue;
        b.tile_start[j] = b.total_tiles;
        b.total_tiles += tiles_of<T>(b.job[j]);
    }
    b.tile_start[b.njobs] = b.total_tiles;
    cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int grid = b.total_tiles < nsm ? b.total_tiles : nsm;
    costagg_batch_kernel<T><<<grid, T::NT, T::BYTES, s>>>(b);
    return cudaGetLastError();
}


template <class T>
cudaError_t launch_one(const CostAggArgs &a, cudaStream_t s)
{
    return launch_dependent(costagg_wta_kernel<T>, dim3(tiles_of<T>(a)), dim3(T::NT), T::BYTES, s, a);
}

template <class T>
double estimate(const CostAggArgs &a, int nsm)
{
    // time ~ waves x per-CTA work per row (producer entries + consumer cells);
    // 32-bit prefixes leave room for fewer row slots and producer warps
    const long ctas = tiles_of<T>(a);
    const long waves = (ctas + nsm - 1) / nsm;
    const double work = (double)T::DS * T::NE + 2.0 * T::XS * T::DS;
    return (double)waves * work * (T::S16 ? 1.0 : 1.15);
}

}  // namespace

cudaError_t costagg_setup()
{
    cudaError_t e = cudaSuccess;
    for (int id = 0; id < kNumTiles && e == cudaSuccess; ++id)
        with_tile(id, [&](auto tag) { e = setup_one<typename decltype(tag)::type>(); });
    return e;
}

int costagg_pick(const CostAggArgs &a, int nsm)
{
    int best = -1;
    double bt = 0;
    for (int id = 0; id < kNumTiles; ++id)
        with_tile(id, [&](auto tag) {
            using T = typename decltype(tag)::type;
            if (!fits<T>(a)) return;
            const double est = estimate<T>(a, nsm);
            if (best < 0 || est < bt) {
                best = id;
                bt = est;
            }
        });
    return best;
}

bool costagg_fits(const CostAggArgs &a, int tile)
{
    bool ok = false;
    with_tile(tile, [&](auto tag) { ok = fits<typename decltype(tag)::type>(a); });
    return ok;
}

cudaError_t launch_costagg_batch(BatchArgs &b, int tile, int nsm, cudaStream_t s)
{
    if (b.njobs < 1 || b.njobs > kMaxBatch) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    with_tile(tile, [&](auto tag) { e = launch_batch_one<typename decltype(tag)::type>(b, nsm, s); });
    return e;
}

cudaError_t launch_costagg(const CostAggArgs &a, cudaStream_t s)
{
    if (a.wy > kMaxWy || a.wy < 0 || a.wx < 0 || a.wx > kMaxWx) return cudaErrorInvalidValue;
    const int tile = a.tile >= 0 ? a.tile : costagg_pick(a, a.num_sms);
    cudaError_t e = cudaErrorInvalidValue;
    with_tile(tile, [&](auto tag) {
        using T = typename decltype(tag)::type;
        if (fits<T>(a)) e = launch_one<T>(a, s);
    });
    return e;
}

}  // namespace stereo
