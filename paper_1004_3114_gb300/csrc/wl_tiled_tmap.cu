// Many passes of one n = 4 binary32 pool in one cooperative launch: the
// lane-tiled bulk-copy pass of wl_tiled_tma.cu (N % 4 == 0 and N coprime to
// 15, so every stride divides 45: 45 lanes x 64 lane times per tile, three
// stages of a warp-specialised ring), with the ring kept across passes and a
// bounded grid barrier between them.
//
// One launch per pass pays, at each pass boundary, for the last CTA's end of
// pass (Eq. 3's scale and the next strides), the grid's completion and the
// release of the next launch before the first bulk copies of the next pass
// can go out: about 9 us per pass on a 2^26-value pool, measured as the part
// of the pass time that does not grow with the pool.  Here every CTA, after
// the barrier, runs the end of pass itself on its own shared-memory copy of
// the state (the same arithmetic in every CTA, as in wl_l2run.cu) while its
// producer warps already copy the next pass's first tiles: their strides
// were drawn a pass ahead, the lane tables for them are built before the
// barrier, and only the consumers' final multiply needs the new scale.
//
// Per pass p: tiles come from counter p mod 3 (zeroed by CTA 0 during the
// pass before), the CTA's sum of squares goes to accumulator set p mod 3,
// and pass p's returned values go to out + p R (the last pass: its first
// last_take).  The ring's mbarriers count their uses across passes; the
// producers end a pass with a stage that carries no tile, and the consumers
// release that stage too, so the next pass finds every stage's use count
// where it expects it.  Every wait is bounded (about a second): a CTA that
// gives up raises the grid's abort flag and WALLACE_ETIMEOUT, stops issuing
// copies, waits (bounded) for its copies in flight and leaves at the next
// barrier with the others.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "wl_common.cuh"
#include "wl_gridsync.cuh"
#include "wl_launch.h"
#include "wl_tma_common.cuh"

namespace {

using namespace wl_tma;

struct MpArgs {
    float *buf[2];
    int cur;
    WlDevState *st;
    WlGridSync *sy;
    int64_t N, Np, R;
    int64_t passes;
    float *out;           // pass p writes its first take values to out + p R (may be null)
    int64_t last_take;    // values the last pass returns (the others return R)
    float mu, sigma;
    double rnu;           // sqrt(2 nu - 1)
};

// Lane tables of a pass whose strides all divide 45 (L = their lcm): J[L + 1],
// span starts spanC[] and, per lane and sub-vector, the slot offset of the
// lane's first value packed with its span (tab layout as in wl_tiled_tma.cu).
// Every thread calls; the caller orders earlier readers before and later
// readers after (barriers).
__device__ void mp_tables(int N32, int L, int T, const int *alpha, const int *m, const int *sb, const int *slot0,
                          const int *SL, int *tab)
{
    int *J = tab;
    int *lanebase = J + (TM_LMAX2 + 1);
    int *spanC = lanebase + 4 * TM_LMAX;
    const int tid = threadIdx.x;
    for (int l = tid; l <= L; l += TM_THREADS) {
        const int qN = tm_divc(N32, L), rN = N32 - qN * L;
        J[l] = l * qN + tm_divc(l * rN + L - 1, L);
    }
    for (int s = tid; s < sb[4]; s += TM_THREADS) {
        const int i = tm_sub<4>(s, sb);
        const int p = s - sb[i], mi = m[i];
        const int qN = tm_divc(N32, mi), rN = N32 - qN * mi;
        spanC[s] = p * qN + tm_divc(p * rN + mi - 1, mi);
    }
    __syncthreads();
    for (int e = tid; e < 4 * L; e += TM_THREADS) {
        const int i = tm_divc(e, L), l = e - i * L;
        const int w = tm_divc(l, m[i]), p = l - w * m[i];
        const int64_t r = (int64_t)alpha[i] * J[l] - (int64_t)w * N32 - spanC[sb[i] + p];
        lanebase[i * TM_LMAX + l] = ((slot0[i] + p * SL[i] + (int)r) << 5) | (sb[i] + p);
    }
}

// The geometry of a pass from its strides: whether they all divide 45, the
// lane count, spans per sub-vector and their slots.
struct MpGeo {
    int L, T, nspans;
    bool tileable;
    int m[4], sb[5], SL[4], slot0[4];
};

__device__ __forceinline__ MpGeo mp_geometry(const int *alpha)
{
    MpGeo g;
    int e3 = 0, e5 = 0;
    g.tileable = true;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int al = alpha[i];
        if (al == 3 || al == 15)
            e3 = max(e3, 1);
        if (al == 9 || al == 45)
            e3 = 2;
        if (al == 5 || al == 15 || al == 45)
            e5 = 1;
        g.tileable &= al == 3 || al == 5 || al == 9 || al == 15 || al == 45;
    }
    g.L = g.tileable ? (e3 == 2 ? 9 : (e3 == 1 ? 3 : 1)) * (e5 ? 5 : 1) : TM_LMAX + 1;
    g.sb[0] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        g.m[i] = g.tileable ? tm_divc(g.L, alpha[i]) : 0;
        g.sb[i + 1] = g.sb[i] + g.m[i];
    }
    g.nspans = g.sb[4];
    g.T = g.tileable ? tm_divc(TM_ETARGET, g.L) : 1;
    g.slot0[0] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        g.SL[i] = (alpha[i] * g.T + 8 + 3) & ~3;   // 16-byte aligned slots; wrap copies need +6
        if (i < 3)
            g.slot0[i + 1] = g.slot0[i] + g.m[i] * g.SL[i];
    }
    g.tileable &= g.nspans <= TM_MAXSPANS;
    return g;
}

