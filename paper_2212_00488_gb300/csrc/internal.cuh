// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stereo {

// Packed per-pixel words written by the support stage and read by the fused
// cost/aggregation kernel:
//   pix = grey | census << 8                       (uint32, bits 14..31 zero)
//   arm = left | right << 8 | up << 16 | down << 24 (uint32, arm lengths)
__host__ __device__ inline uint32_t pack_arm(int hm, int hp, int vm, int vp)
{
    return (uint32_t)hm | ((uint32_t)hp << 8) | ((uint32_t)vm << 16) | ((uint32_t)vp << 24);
}

// Arm words of the fused kernel, row quads interleaved: the word of row r and
// column x sits at ((r / 4) X + x) 4 + r % 4, so one 16-byte load fetches a
// column's words of four consecutive rows. Row r holds the left/right arms of
// row r (low half) and the up/down arms of row r - wy (high half); rows run
// to Y + wy - 1, rounded up to whole quads.
__host__ __device__ inline size_t armc_index(int r, int x, int X)
{
    return ((size_t)(r >> 2) * X + x) * 4 + (r & 3);
}
inline size_t armc_words(int X, int Y, int wy) { return (size_t)X * (size_t)((Y + wy + 3) / 4) * 4; }

// Tile shape of the fused kernel (see costagg.cu).
constexpr int kRing = 64;      // V-prefix ring depth: 2*wy + 2 <= 64
constexpr int kMaxWy = 31;
constexpr int kMaxWx = 141;    // the largest W_x of Table I

struct CostAggArgs {
    const uint32_t *pix_l, *pix_r;   // [Y][X]
    const uint32_t *arm_l, *arm_r;   // [Y][X]
    const uint32_t *armc_l, *armc_r; // armc_words(X, Y, wy), laid out by armc_index
    uint32_t *key_l, *key_r;         // [Y][X] min over d of (CA << 8 | d); preset to ~0
    const uint32_t *lut_ad;          // [256] quantised AD cost (Eq. 4) by |grey difference|
    const uint32_t *lut_mc;          // [8] quantised census cost (Eq. 5) by Hamming distance
    uint32_t *err;                   // set to nonzero when a bounded wait gives up
    uint32_t wait_limit;             // polls per mbarrier wait before giving up
    int X, Y, D;
    int wx, wy;
    uint32_t P;                      // cost of a match outside the image
    int tile;                        // tile shape id, -1 = pick from the shape
    int num_sms;                     // SMs of the device (for the pick)
};

// Programmatic dependent launch between the kernels of a frame: a kernel
// launched with launch_dependent may start while the previous kernel on the
// stream is still running; it calls pdl_wait() before it touches anything
// that kernel writes (the wait returns once the previous grid has completed
// and its memory is visible). Every kernel calls pdl_trigger() first, so the
// next one can be scheduled as soon as all of its CTAs are running.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Number of tile shapes of the fused kernel (ids 0 .. kNumTiles-1).
constexpr int kNumTiles = 9;
int costagg_pick(const CostAggArgs &a, int nsm);
bool costagg_fits(const CostAggArgs &a, int tile);

// A batch of frames for the persistent form of the fused kernel.
constexpr int kMaxBatch = 32;
struct BatchArgs {
    int njobs;
    int total_tiles;                  // filled by the launcher
    int tile_start[kMaxBatch + 1];    // first tile of each job (filled by the launcher)
    CostAggArgs job[kMaxBatch];       // every job's err points at the same word
    uint32_t *counter;                // tile counter, zeroed by the launcher
};
// Launches the persistent batch kernel with tile shape `tile` on nsm CTAs.
cudaError_t launch_costagg_batch(BatchArgs &b, int tile, int nsm, cudaStream_t s);

// Differentiable form (diff.cu): B pairs of W x H at processed resolution.
struct DiffArgs {
    int B, W, H, D;
    const float *left, *right;         // [B][H][W][3] float RGB on [0, 1]
    const uint8_t *left_u8, *right_u8; // [B][H][W][3] uint8 RGB the frozen supports come from
    const float *theta;                // [4] w_AD, w_MC, lambda_AD, lambda_MC
    float tau;
    float *dhat;                       // [B][H][W]
    float *stats;                      // [B][H][W][2] softmax max and sum (written by forward)
    const float *grad_dhat;            // backward only
    float *grad_left, *grad_right;     // backward only, [B][H][W][3]
    float *grad_theta;                 // backward only, [4]
    int backward;
    void *ws;                          // diff_workspace_bytes(W, H, wy, B, D) bytes
    uint32_t *err;
    int wx, wy, tc;
};
size_t diff_workspace_bytes(int X, int Y, int wy, int B, int D);
// Sets the differentiable kernels' attributes on the current device (call
// before diff_run and outside any stream capture).
cudaError_t diff_setup();
cudaError_t diff_run(const DiffArgs &a, cudaStream_t s);

// Launchers (each returns the launch error, cudaSuccess on success).
cudaError_t launch_grey(const uint8_t *rgb_l, const uint8_t *rgb_r, uint8_t *g_l, uint8_t *g_r,
                        int W, int H, cudaStream_t s);
// Grey of both images and its Eq. 2 downscale, with the full-resolution grey
// of the left image (what the scale-up reads): one launch when W is a
// multiple of 4 and the RGB rows are word-aligned (gf_r is then not written),
// else grey_kernel and downscale_kernel. Adds the kernels launched to
// *launches.
cudaError_t launch_grey_down(const uint8_t *rgb_l, const uint8_t *rgb_r, uint8_t *gf_l, uint8_t *gf_r,
                            uint8_t *s_l, uint8_t *s_r, int W, int H, cudaStream_t s, int *launches);
cudaError_t launch_downscale(const uint8_t *g_l, const uint8_t *g_r, uint8_t *s_l, uint8_t *s_r,
                             int W, int H, cudaStream_t s);
// Also presets the WTA keys of both bases to ~0 and clears the fused
// kernel's error word for this frame.
cudaError_t launch_support(const uint8_t *g_l, const uint8_t *g_r, uint32_t *pix_l, uint32_t *pix_r,
                           uint32_t *arm_l, uint32_t *arm_r, uint32_t *armc_l, uint32_t *armc_r,
                           uint32_t *key_l, uint32_t *key_r, uint32_t *err, int X, int Y, int wx, int wy,
                           int tc, cudaStream_t s);
cudaError_t launch_costagg(const CostAggArgs &a, cudaStream_t s);
cudaError_t launch_refine(const uint32_t *key_l, const uint32_t *key_r, const uint8_t *grey_l,
                          int X, int Y, int T, int fill_mode, uint8_t *dl, uint8_t *dr, uint8_t *gcp,
                          uint8_t *dm, float *dplus, cudaStream_t s);
// The downscaling path's Steps 6-8 in one kernel: the maps and dplus of
// launch_refine, and the full-resolution disparity in out.
cudaError_t launch_refine_up(const uint32_t *key_l, const uint32_t *key_r, const uint8_t *grey_low,
                             const uint8_t *grey_full, int X, int Y, int W, int H, int T, int fill_mode, uint8_t *dl,
                             uint8_t *dr, uint8_t *gcp, uint8_t *dm, float *dplus, float *out, cudaStream_t s);
cudaError_t launch_unpack_planes(const uint32_t *pix, const uint32_t *arm, uint8_t *grey,
                                 uint8_t *census, uint32_t *arms, int X, int Y, cudaStream_t s);


// One-time per-device function attributes (large dynamic shared memory);
// call with the device current.
cudaError_t costagg_setup();
cudaError_t refine_setup();

}  // namespace stereo
