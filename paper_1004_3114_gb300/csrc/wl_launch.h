// Host-side launchers of the Wallace generator kernels (internal to the
// library; the public interface is include/wallace.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct WlDevState;

// Arguments of one pass.  Pools hold n sub-vectors of length N at row pitch
// Np elements.  Pool values with logical index q in [w0, w1) are also written,
// mapped to mu + sigma*y, to out[q - w0] (the returned prefix of the pass).
struct WlPassArgs {
    const void *src;
    void *dst;
    int n;
    int64_t N, Np, nu;
    WlDevState *st;
    void *out;
    int64_t w0, w1;
    double mu, sigma;
    int64_t pass;   // passes completed before this one (selects its strides' slot)
};

// opts: bit 0 -- the Wilson-Hilferty chi-squared sample instead of Eq. 3's;
//       bit 1 -- a random sign pattern per pass (matrix A D_k)
cudaError_t wl_launch_init(void *pool, int fp64, int n, int64_t N, int64_t Np, uint32_t seed,
                           uint32_t stream_id, WlDevState *st, int sm_count, cudaStream_t stream,
                           int opts = 0);

// Box-Muller refill of the current pool for restart r = 1, 2, ... (Section 5)
cudaError_t wl_launch_restart(void *pool, int fp64, int n, int64_t N, int64_t Np, uint32_t seed,
                              uint32_t stream_id, int64_t r, WlDevState *st, int sm_count,
                              cudaStream_t stream);

// direct strided gather from global memory, any n, N, either precision
// Two-phase pass for stride sets with strides up to WL_TWOPHASE_MAX_STRIDE
// (binary32; half of it for binary64 pools): un-stride into `scratch` (n rows
// of pitch Np), then stream the transform (2 launches).
#define WL_TWOPHASE_MAX_STRIDE 16384
cudaError_t wl_launch_twophase(const WlPassArgs &a, void *scratch, int fp64, int sm_count, cudaStream_t stream);
cudaError_t wl_launch_gather(const WlPassArgs &a, int fp64, int sm_count, cudaStream_t stream);

// out[k] = mu + sigma * pool[pos + k], k < count (values already produced)
cudaError_t wl_launch_drain(const void *pool, int fp64, int64_t N, int64_t Np, int64_t pos,
                            int64_t count, void *out, double mu, double sigma, int sm_count,
                            cudaStream_t stream);

// lane-tiled gather staged through shared memory (binary32, n = 4)
bool wl_tiled_supported(int n, int64_t N, int fp64);
cudaError_t wl_launch_tiled(const WlPassArgs &a, int sm_count, cudaStream_t stream);

// warp-specialised lane-tiled gather with bulk (TMA) copies into a stage ring
// (binary32, n = 4, N a multiple of 4)
bool wl_tma_supported(int n, int64_t N, int fp64, int sm_count);
// signs: the generator draws a sign pattern per pass (matrix A D_k)
cudaError_t wl_launch_tma(const WlPassArgs &a, int sm_count, int signs, cudaStream_t stream);

// the same for n = 8 (binary32, N a multiple of 4 and coprime to 105: 315
// lanes, eight sub-vectors per stage)
bool wl_tma8_supported(int n, int64_t N, int fp64);
// the pass's returned values, for pools above 64 MB, come from a second
// kernel (streaming, after the pass): whether this pass takes it
bool wl_tma8_return_kernel(const WlPassArgs &a);
cudaError_t wl_launch_tma8(const WlPassArgs &a, int sm_count, int signs, cudaStream_t stream);
// that second kernel alone: out[q - w0] = mu + sigma dst[q] over [w0, w1)
cudaError_t wl_launch_t8_return(const WlPassArgs &a, int sm_count, cudaStream_t stream);

// n = 8 on clusters of two CTAs, each with four of the eight sub-vectors of
// a 315-lane x 16-lane-time tile (the same pools as wl_tma8_supported, when
// a cluster of two fits the device); the grid is every resident cluster
bool wl_tma8c_supported(int n, int64_t N, int fp64);
// whether WALLACE_VARIANT_TILED (and AUTO) takes the cluster form for this pool
bool wl_tma8c_preferred(int n, int64_t N, int fp64);
int wl_tma8c_grid();
cudaError_t wl_launch_tma8c(const WlPassArgs &a, int sm_count, int signs, cudaStream_t stream);

// many passes of one n = 4 or 8 binary32 pool of at most 2^23 values in one
// cooperative launch of `grid` CTAs (capped at what can be resident), with a
// bounded grid barrier per pass (pools that stay in L2 between passes); every
// stride must satisfy (alpha + 1) N < 2^32 (max_stride: the largest the pool
// can draw).  `sync` is a device block of wl_l2run_sync_bytes() bytes, zeroed
// here before the launch.  The pool is in buffer `cur` of (buf0, buf1); pass k
// writes its values [0, take_k) to out + k R (take_k = R, last_take for the
// last).  The final pool is in the other buffer when `passes` is odd.
// signs: the generator draws a sign pattern per pass (matrix A D_k).
bool wl_l2run_supported(int n, int64_t N, int fp64, int64_t max_stride);
size_t wl_l2run_sync_bytes();
int wl_l2run_grid(int64_t nu, int sm_count);
// pools AUTO sends to it: above the shared-memory size, at most this many values
#define WL_L2RUN_AUTO_MAX_VALUES ((int64_t)1 << 22)
cudaError_t wl_launch_l2run(void *buf0, void *buf1, int cur, int n, int64_t N, int64_t Np, WlDevState *st,
                            void *sync, int64_t passes, int64_t R, int64_t last_take, void *out, double mu,
                            double sigma, int grid, int signs, cudaStream_t stream);

// whole pool resident in shared memory for `passes` passes in one launch.
// Pass k (0-based) writes its values [0, take_k) to out + out_off_k where
// take_k = R for k < passes-1 and last_take for the final pass.
bool wl_fused_supported(int n, int64_t N, int fp64, int64_t *smem_bytes);
cudaError_t wl_launch_fused(void *pool_cur, void *pool_other, int fp64, int n, int64_t N,
                            int64_t Np, WlDevState *st, int64_t passes, int64_t R,
                            int64_t last_take, void *out, double mu, double sigma,
                            cudaStream_t stream);
