// lbm_pf.cu -- kernels and C ABI (include/lbm_pf.h) of the GB300 phase-field
// lattice Boltzmann library (Liang et al., arXiv:1710.09541, Sec. II).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include <cudaTypedefs.h>

#include "lbm_kernels.cuh"
#include "lbm_pf.h"
#include "lbm_store.cuh"

using namespace lbmpf;

namespace {

// ---------------------------------------------------------------------------
// The fused step kernel.  With FP32 storage one thread per node of a TX x TY
// tile; with 16-bit storage each thread takes LBM_NPT16 nodes of a taller
// tile (step_tile16).  Phase 1 pulls f_i and g_i of the node, forms phi
// (Eq. 12) and writes it to shared memory; threads also form phi on the
// one-node ring around the tile (each ring node pulls its own 9 f_i, mostly
// L2 hits as neighbouring tiles read the same lines).  Phase 2 takes the
// stencils of Eqs. 27-28 from shared memory, recovers rho, mu_phi, F, u, p
// (Eqs. 5-7, 13, 19, 22), collides f and g (Eqs. 8-11, 15-20) and stores both
// sets at the node's own address.
//
// FIELDS = true evaluates the same formulas but writes phi, rho, ux, uy, p
// as doubles instead of colliding (used by lbm_get_fields and lbm_diag).
// CHK = true adds the non-finite test of each node (handles that asked for
// checks).
// ---------------------------------------------------------------------------
#ifndef LBM_STEP_TX
#define LBM_STEP_TX 32
#endif
#ifndef LBM_STEP_TY
#define LBM_STEP_TY 4
#endif
#ifndef LBM_STEP_MINB
#define LBM_STEP_MINB 0
#endif
// Debug build (LBM_DEBUG_CHECKS = 1, the library liblbm_pf_debug.so): the
// step checks every neighbour row and column and every shared-memory slot it
// computes, records an out-of-range one as bit 4 of the error flag (the call
// returns LBM_ERR_CUDA) and skips it, and poisons the tile's phi slots with
// NaN before filling them.  It stands in for a sanitizer: the arithmetic is
// the same, so results equal the release library's bit for bit.
#ifndef LBM_DEBUG_CHECKS
#define LBM_DEBUG_CHECKS 0
#endif
#if LBM_DEBUG_CHECKS
__device__ __forceinline__ bool nbr_in_range(const Nbr& q, int nx, int ny) {
    const int last = (ny - 1) * nx;
    auto row = [&](int r) { return r >= 0 && r <= last && r % nx == 0; };
    auto col = [&](int c) { return c >= 0 && c < nx; };
    return row(q.r0) && row(q.rm) && row(q.rp) && col(q.x) && col(q.xm) && col(q.xp);
}
#endif

// load (phi u) of the previous step with the node's pulls instead of just
// before the collision
#ifndef LBM_EARLY_PHIU
#define LBM_EARLY_PHIU 1
#endif
// L2 prefetch distance of the FP32 step kernel in tiles, per 10 SMs (0: off);
// 30 = 3 tiles of 32 x 4 per SM, about a third of a resident wave at 10
// blocks/SM.  With the alternating tile order, one grid per process (MLUPS at
// 1 / 1.5 / 2 / 3 / 4 / 5 tiles per SM): 2048^2 39.7 / 40.3 / 40.6 / 40.7 /
// 40.3 / 39.9 k, impact 2400 x 2400 38.6 / 39.2 / 39.7 / 39.9 / 39.6 / 39.3 k,
// impact 2400 x 600 37.1 / 37.5 / 37.7-37.8 / 37.7 / 37.5 / 37.2 k.  (Before
// that order, in one process over several grids, 2 to 2.5 had been best.)
#ifndef LBM_PREFETCH_PER10SM
#define LBM_PREFETCH_PER10SM 30
#endif
// prefetch distance of the 16-bit step kernels, in tiles per 10 SMs: periodic
// and walled grids.  Measured with one grid per process (FP16 MLUPS at 10 /
// 15 / 20 / 30 / 40): 2048^2 56.3 / 57.0 / 57.2 / 56.3 / 55.4 k, 3072^2 59.5 /
// 60.8 / 61.0 / 60.7 / 59.4 k, 1792^2 54.9 / 55.7 / 56.1 / 55.6 / 54.5 k;
// impact 2400 x 2400 55.6 / 55.6 / 55.2 / 53.6 / 52.3 k (per-thread requests).
// With the tensor-map prefetch, at 10 / 20 / 30 (walls 10 / 15 / 30): 2048^2
// 59.8 / 60.7 / 60.6 k, 3072^2 62.8 / 64.3 / 64.7 k, impact 2400 x 2400
// 58.5 / 58.7 / 56.8 k
#ifndef LBM_PREFETCH16_PER10SM
#define LBM_PREFETCH16_PER10SM 20
#endif
#ifndef LBM_PREFETCH16_WALLS_PER10SM
#define LBM_PREFETCH16_WALLS_PER10SM 15
#endif
// prefetch with 16-bit storage too.  With one node per thread the requests
// cost more than they hid (FP16 at 2048^2 47.6 k -> 45.5 k MLUPS); with two
// nodes per thread they pay (54.6 k -> 57.6 k)
#ifndef LBM_PREFETCH_16
#define LBM_PREFETCH_16 1
#endif
// alternate the tiles' order from step to step (the step reading buffer 1
// walks them backwards)
#ifndef LBM_ALTERNATE_ORDER
#define LBM_ALTERNATE_ORDER 1
#endif
// steps whose algorithmic traffic is below this many tenths of the L2 size
// run without the prefetch: FP32 and 16-bit storage.  With the alternating
// tile order, measured with one grid per process (MLUPS, prefetch on / off):
// FP32 1024^2 (168 MB per step) 38.6 / 39.6 k, FP32 impact 2400 x 600
// (230 MB) 37.8 / 36.9 k; FP16 1536^2 (217 MB) 52.2 / 55.5 k, impact
// 2400 x 1200 (265 MB) 53.2 / 55.3 k, 1792^2 (295 MB) 56.1 / 55.4 k, impact
// 2400 x 1500 (331 MB) 54.9 / 54.9 k, impact 2400 x 1600 (353 MB) 54.8 /
// 54.1 k, 2048^2 (386 MB) 57.3 / 56.5 k.  The 16-bit threshold sits between
// 265 and 295 MB.
#ifndef LBM_PREFETCH_L2X10
#define LBM_PREFETCH_L2X10 15
#endif
#ifndef LBM_PREFETCH16_L2X10
#define LBM_PREFETCH16_L2X10 21
#endif
// the same threshold for 16-bit steps that prefetch through tensor maps, whose
// requests cost almost no issue slots (one grid per process, FP16 MLUPS,
// prefetch on / off): impact 2400 x 600 (133 MB) 54.8 / 56.0 k, 1536^2
// (217 MB) 55.2 / 55.1 k, impact 2400 x 1200 (265 MB) 56.3 / 54.6 k
#ifndef LBM_PREFETCH16_TMA_L2X10
#define LBM_PREFETCH16_TMA_L2X10 15
#endif
// One TX x TY tile with origin (x0, y0): the body shared by the single-case
// step kernel and the batched kernel (so both give the same bits).
template <int TX, int TY, bool FIELDS, int WALLS, int ST, bool CHK>
__device__ __forceinline__ void step_tile(float (*sphi)[TX + 2], const float* __restrict__ fs,
                                          const float* __restrict__ gs, float* __restrict__ fd,
                                          float* __restrict__ gd, float* __restrict__ phiu,
                                          unsigned int* __restrict__ flag, double* __restrict__ out,
                                          int nx, int ny, Model m, int x0, int y0) {
    if (WALLS == 0) m.walls = 0;  // WALLS == 1 keeps the kind of top (wall or open)
    const int wfold = WALLS >= 0 ? WALLS : m.walls;  // y folding: wrap (0) or clamp
    const size_t N = (size_t)nx * ny;
    const int N32 = (int)N;  // 20 N < 2^31 (checked at create): 32-bit offsets
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < nx) && (y < ny);

    // Phase 1: the node's own pulls (f for phi, g for the collision after the
    // barrier), then phi on the ring around the tile, one ring node per
    // thread on the first threads so only the first warps take that path.
    float f[9], g[9];
    Nbr q;
#if LBM_EARLY_PHIU
    float2 prev = make_float2(0.f, 0.f);
#endif
#if LBM_DEBUG_CHECKS
    // poison the tile's phi slots: a slot that phase 1 fails to write reaches
    // the stencil as NaN and trips the non-finite check
    for (int k = ty * TX + tx; k < (TY + 2) * (TX + 2); k += TX * TY)
        (&sphi[0][0])[k] = __int_as_float(0x7fc00000);
    __syncthreads();
#endif
    if (active) {
        q = make_nbr<WALLS>(x, y, nx, ny, m.walls);
#if LBM_DEBUG_CHECKS
        if (!nbr_in_range(q, nx, ny)) {  // record, and pull node 0 instead
            atomicOr(flag, 4u);
            q = make_nbr<WALLS>(0, 0, nx, ny, m.walls);
        }
#endif
#if LBM_EARLY_PHIU
        if (!FIELDS) prev = make_float2(phiu[q.r0 + x], phiu[N32 + q.r0 + x]);
#endif
        pull18<ST, WALLS>(fs, gs, N32, q, f, g);
        sphi[ty + 1][tx + 1] = Pop<ST>::phi_of(f);
    } else {
        sphi[ty + 1][tx + 1] =
            phi_at_st<ST, WALLS>(fs, N32, fold_x(x, nx), fold_y(y, ny, wfold), nx, ny, m.walls);
    }
    for (int r = ty * TX + tx; r < Ring<TX, TY>::count; r += TX * TY) {
        int lx, ly;
        Ring<TX, TY>::pos(r, lx, ly);
#if LBM_DEBUG_CHECKS
        const int fx = fold_x(x0 + lx, nx), fy = fold_y(y0 + ly, ny, wfold);
        if (lx < -1 || lx > TX || ly < -1 || ly > TY || fx < 0 || fx >= nx || fy < 0 || fy >= ny) {
            atomicOr(flag, 4u);
            continue;
        }
#endif
        sphi[ly + 1][lx + 1] = phi_at_st<ST, WALLS>(fs, N32, fold_x(x0 + lx, nx),
                                                    fold_y(y0 + ly, ny, wfold), nx, ny, m.walls);
    }
    __syncthreads();
    if (!active) return;

    const int lx = tx + 1, ly = ty + 1;
    const float phi = sphi[ly][lx];
    const Stencil st = stencil(phi, sphi[ly][lx + 1], sphi[ly][lx - 1], sphi[ly + 1][lx],
                               sphi[ly - 1][lx], sphi[ly + 1][lx + 1], sphi[ly + 1][lx - 1],
                               sphi[ly - 1][lx - 1], sphi[ly - 1][lx + 1]);
    const Macro M = macro_from(m, Pop<ST>::gmom(g), phi, st.gx, st.gy, st.lap);
    const int n32 = q.r0 + x;

    if (FIELDS) {
        out[n32] = phi;
        out[N + n32] = M.rho;
        out[2 * N + n32] = M.ux;
        out[3 * N + n32] = M.uy;
        out[4 * N + n32] = M.p;
        return;
    }
    // one test: a NaN or Inf in any of phi, u, p makes the sum non-finite;
    // reported after the stores, so the branch does not split the update
    bool bad = false;
    if constexpr (CHK) bad = m.check_nonfinite && !isfinite(add(add(phi, M.ux), add(M.uy, M.p)));

#if !LBM_EARLY_PHIU
    const float2 prev = make_float2(phiu[n32], phiu[N32 + n32]);
#endif
    const float2 now = collide_st<ST>(m, f, g, phi, st, M, prev);
    phiu[n32] = now.x;
    phiu[N32 + n32] = now.y;
    Pop<ST>::stfg(fd, gd, N32, n32, f, g, phi);
    if constexpr (CHK)
        if (bad) report_nonfinite(flag);
}

// One TX x (NPT TY) tile with 16-bit storage: each of the TX x TY threads
// takes NPT nodes, in rows ty, ty + TY, ...  Between the two phases a node
// holds its nine raw code words rather than 18 converted values, so that two
// nodes per thread fit the register budget; the codes are converted where they
// are used.  The arithmetic is step_tile's (same functions, same order), so a
// node gets the same bits whichever body, tile shape or kernel steps it.
#ifndef LBM_NPT16
#define LBM_NPT16 2
#endif
template <int TX, int TY, int NPT, int WALLS, int ST, bool CHK>
__device__ __forceinline__ void step_tile16(float (*sphi)[TX + 2], const void* __restrict__ fs,
                                            const void* __restrict__ gs, void* __restrict__ fd,
                                            void* __restrict__ gd, float* __restrict__ phiu,
                                            unsigned int* __restrict__ flag, int nx, int ny, Model m,
                                            int x0, int y0) {
    constexpr bool BR = (WALLS < 0) || LBM_WALL_BRANCH;
    constexpr int TH = TY * NPT;
    if (WALLS == 0) m.walls = 0;  // WALLS == 1 keeps the kind of top (wall or open)
    const int wfold = WALLS >= 0 ? WALLS : m.walls;  // y folding: wrap (0) or clamp
    const int N = nx * ny;  // 20 N < 2^31 (checked at create): 32-bit offsets
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx;
    unsigned int w[NPT][9];
    float f0[NPT];
    unsigned short g0[NPT];
    float2 prev[NPT];
    int n[NPT];
    bool act[NPT];
#if LBM_DEBUG_CHECKS
    for (int k = ty * TX + tx; k < (TH + 2) * (TX + 2); k += TX * TY)
        (&sphi[0][0])[k] = __int_as_float(0x7fc00000);
    __syncthreads();
#endif
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int ly = ty + TY * j, y = y0 + ly;
        act[j] = (x < nx) && (y < ny);
        n[j] = 0;
        prev[j] = make_float2(0.f, 0.f);
        if (act[j]) {
            Nbr q = make_nbr<WALLS>(x, y, nx, ny, m.walls);
#if LBM_DEBUG_CHECKS
            if (!nbr_in_range(q, nx, ny)) {  // record, and pull node 0 instead
                atomicOr(flag, 4u);
                q = make_nbr<WALLS>(0, 0, nx, ny, m.walls);
            }
#endif
            n[j] = q.r0 + q.x;
            prev[j] = make_float2(phiu[n[j]], phiu[N + n[j]]);
            pull_words16<ST, BR, true>(fs, gs, N, q, w[j], f0[j], g0[j]);
            float h[9];
            codes_f<ST>(w[j], f0[j], h);
            sphi[ly + 1][tx + 1] = Pop<ST>::phi_of(h);
        } else {
            sphi[ly + 1][tx + 1] =
                phi_at_st<ST, WALLS>(fs, N, fold_x(x, nx), fold_y(y, ny, wfold), nx, ny, m.walls);
        }
    }
    for (int r = ty * TX + tx; r < Ring<TX, TH>::count; r += TX * TY) {
        int lx, ly;
        Ring<TX, TH>::pos(r, lx, ly);
#if LBM_DEBUG_CHECKS
        const int fx = fold_x(x0 + lx, nx), fy = fold_y(y0 + ly, ny, wfold);
        if (lx < -1 || lx > TX || ly < -1 || ly > TH || fx < 0 || fx >= nx || fy < 0 || fy >= ny) {
            atomicOr(flag, 4u);
            continue;
        }
#endif
        sphi[ly + 1][lx + 1] = phi_at_st<ST, WALLS>(fs, N, fold_x(x0 + lx, nx),
                                                    fold_y(y0 + ly, ny, wfold), nx, ny, m.walls);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        if (!act[j]) continue;
        const int lx = tx + 1, ly = ty + TY * j + 1;
        float h[9], k[9];
        codes_f<ST>(w[j], f0[j], h);
        codes_g<ST>(w[j], g0[j], k);
        const float phi = sphi[ly][lx];
        const Stencil st = stencil(phi, sphi[ly][lx + 1], sphi[ly][lx - 1], sphi[ly + 1][lx],
                                   sphi[ly - 1][lx], sphi[ly + 1][lx + 1], sphi[ly + 1][lx - 1],
                                   sphi[ly - 1][lx - 1], sphi[ly - 1][lx + 1]);
        const Macro M = macro_from(m, Pop<ST>::gmom(k), phi, st.gx, st.gy, st.lap);
        bool bad = false;
        if constexpr (CHK) bad = m.check_nonfinite && !isfinite(add(add(phi, M.ux), add(M.uy, M.p)));
        const float2 now = collide_code<Pop<ST>>(m, h, k, phi, st, M, prev[j]);
        phiu[n[j]] = now.x;
        phiu[N + n[j]] = now.y;
        Pop<ST>::stfg(fd, gd, N, n[j], h, k, phi, m.seed);
        if constexpr (CHK)
            if (bad) report_nonfinite(flag);
    }
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The same prefetch through tensor maps: one thread of the block asks L2 for
// a whole box of rows of every plane with one bulk tensor prefetch per map
// (cp.async.bulk.prefetch.tensor; it writes no shared memory and waits on
// nothing), instead of one request per thread with its own address.  The maps
// of a handle's two population buffers and of (phi u) are encoded on the host
// (encode_pf_maps); pm.on = 0 keeps the per-thread requests.
// Measured with one grid per process (MLUPS, tensor maps / per-thread
// requests): FP16 2048^2 60.7 / 56.8 k, 3072^2 64.3 / 60.7 k, 1792^2 59.6 /
// 55.7 k, impact 2400 x 2400 58.7 / 55.6 k: the 16-bit step is bound by
// instruction issue, and the per-thread requests (a division by the grid
// width and an address per thread) were about 4% of its instructions.  FP32
// 2048^2 40.4 / 40.9 k, impact 2400 x 600 38.1 / 37.9 k, 2400 x 2400 40.1 /
// 40.1 k: the FP32 step is bound by DRAM and keeps the per-thread requests
// (LBM_TMA_PREFETCH32).
#ifndef LBM_TMA_PREFETCH
#define LBM_TMA_PREFETCH 1
#endif
#ifndef LBM_TMA_PREFETCH32
#define LBM_TMA_PREFETCH32 0
#endif
struct PfMaps {
    CUtensorMap pop[3];  // FP32: the 9 f planes, the 9 g planes; 16-bit: the 8 word planes, f_0, g_0
    CUtensorMap phiu;    // the two (phi u) planes
    int on;
};
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* m, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(m)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* m, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(m)),
                 "r"(x), "r"(y)
                 : "memory");
}
// tile (bx, by) of TX x TY nodes: the boxes start at column bx*TX (a multiple
// of 32 elements, so 16-byte aligned) and at row by*TY - 1, clamped to 0 (the
// top tile row then misses its wrapped halo row, which only costs a miss)
template <int TY, int ST>
__device__ __forceinline__ void prefetch_tile_maps(const PfMaps& pm, int x0, int by) {
    const int y = by * TY > 0 ? by * TY - 1 : 0;
    if constexpr (ST == ST_FP32) {
        tma_prefetch_3d(&pm.pop[0], x0, y, 0);
        tma_prefetch_3d(&pm.pop[1], x0, y, 0);
    } else {
        tma_prefetch_3d(&pm.pop[0], x0, y, 0);
        tma_prefetch_2d(&pm.pop[1], x0, y);
        tma_prefetch_2d(&pm.pop[2], x0, y);
    }
    tma_prefetch_3d(&pm.phiu, x0, by * TY, 0);
}

// Ask L2 for the rows tile (bx, by) of TX x TY nodes will pull: rows
// by*TY - 1 .. by*TY + TY of the population planes and the TY rows of (phi u),
// from column bx*TX (one request per row and plane, one per thread of the NT
// threads).  Called by a block for the tile that starts about a fifth of a
// resident wave after it, so those DRAM reads are in flight while the current
// tiles compute: the step is bound by load latency, and a prefetch holds no
// register and no shared memory.
template <int TX, int TY, int NT, int ST>
__device__ __forceinline__ void prefetch_tile(const void* fs, const void* gs, const float* phiu,
                                              int nx, int ny, int wfold, int bx, int by) {
    constexpr int NP = Pop<ST>::PLANES;
    constexpr int L = (TX + 31) / 32;  // 128-byte lines per tile row of 4-byte entries
    constexpr int NREQ = (NP * (TY + 2) + 2 * TY) * L;
    const int N = nx * ny;
#pragma unroll
    for (int t0 = threadIdx.y * TX + threadIdx.x; t0 < NREQ; t0 += NT) {
        const int t = t0 / L, line = t0 - t * L;
        const int x0 = bx * TX + 32 * line;
        if (x0 >= nx) continue;
        if (t < NP * (TY + 2)) {
            const int plane = t / (TY + 2), r = t - plane * (TY + 2);
            const int idx = fold_y(by * TY - 1 + r, ny, wfold) * nx + x0;
            prefetch_l2(Pop<ST>::plane_addr(fs, gs, N, plane, idx));
        } else {
            const int k = t - NP * (TY + 2), yy = by * TY + (k % TY);
            if (yy < ny) prefetch_l2(phiu + ((k / TY) * N + yy * nx + x0));
        }
    }
}

// Resident blocks per SM each step kernel is compiled for (its register
// budget), measured per instantiation with 32 x 4 tiles at 2048^2 (2400 x 600
// for walls), MLUPS at 8 / 9 / 10 blocks:
//   FP32 periodic 38.7 / 38.6 / 39.4 k; 16-bit periodic 46.5 / 47.6 / 43.6 k;
//   16-bit walls 41.2 / 42.1 / 42.7 k (before the source-folded collision);
//   FP32 walls 32.5 / 33.0 k at 8 / 9 (10 spills), 16-bit periodic 49.4 k at 9
//   against 44.9 k at 10 (with it).  With two nodes per thread the 16-bit
//   kernels take 1024 threads per SM (64 registers): 57.6 k at 2048^2, against
//   56.6 k at 7 blocks (72 registers) and 53.6 k at 10 (spills).
// LBM_STEP_MINB > 0 overrides all of them.
template <bool FIELDS, int WALLS, int ST, int NT>
constexpr int step_minb() {
    if (LBM_STEP_MINB > 0) return LBM_STEP_MINB;
    if (FIELDS) return 8;
    if (ST == ST_FP32) return WALLS == 0 ? 10 : 9;
    if (LBM_NPT16 > 1) return 1024 / NT;  // two nodes per thread: 64 registers, no spills
    return WALLS == 0 ? 9 : 10;
}

// nodes per thread of a step kernel: LBM_NPT16 for 16-bit steps, else 1
template <bool FIELDS, int ST>
__host__ __device__ constexpr int step_npt() {
    return (!FIELDS && ST != ST_FP32) ? LBM_NPT16 : 1;
}

template <int TX, int TY, bool FIELDS, int WALLS, int ST, bool CHK = false>
__global__ void __launch_bounds__(TX* TY, (step_minb<FIELDS, WALLS, ST, TX * TY>()))
    k_step(const float* __restrict__ fs, const float* __restrict__ gs, float* __restrict__ fd,
           float* __restrict__ gd, float* __restrict__ phiu, unsigned int* __restrict__ flag,
           double* __restrict__ out, int nx, int ny, Model m, int pf_ahead, int rev,
           const __grid_constant__ PfMaps pm) {
    constexpr int NPT = step_npt<FIELDS, ST>();
    __shared__ float sphi[TY * NPT + 2][TX + 2];
    // rev = 1 walks the tiles in the reverse order (block (0, 0) takes the last
    // tile): alternate steps meet first the tiles the previous step wrote last,
    // while they are still in L2
    const int bx = rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int by = rev ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    griddep_wait();
    griddep_launch();
    if constexpr (!FIELDS && (ST == ST_FP32 || LBM_PREFETCH_16)) {
        if (pf_ahead > 0 && (!pm.on || (threadIdx.x == 0 && threadIdx.y == 0))) {
            const int lin = blockIdx.y * gridDim.x + blockIdx.x + pf_ahead;
            if (lin < gridDim.x * gridDim.y) {
                int px = lin % gridDim.x, py = lin / gridDim.x;
                if (rev) {
                    px = gridDim.x - 1 - px;
                    py = gridDim.y - 1 - py;
                }
                if (pm.on)
                    prefetch_tile_maps<TY * NPT, ST>(pm, px * TX, py);
                else
                    prefetch_tile<TX, TY * NPT, TX * TY, ST>(fs, gs, phiu, nx, ny,
                                                             WALLS >= 0 ? WALLS : m.walls, px, py);
            }
        }
    }
    if constexpr (NPT > 1 || (!FIELDS && ST != ST_FP32))
        step_tile16<TX, TY, NPT, WALLS, ST, CHK>(sphi, fs, gs, fd, gd, phiu, flag, nx, ny, m,
                                                 bx * TX, by * TY * NPT);
    else
        step_tile<TX, TY, FIELDS, WALLS, ST, CHK>(sphi, fs, gs, fd, gd, phiu, flag, out, nx, ny, m,
                                                  bx * TX, by * TY);
}

// ---------------------------------------------------------------------------
// Initial state.  The canonical (pre-collision) state is f_i = f_i^eq(phi0,u0)
// (Eq. 9) and g_i = g_i^eq(p0, rho(phi0), u0) (Eqs. 13, 16, 17).  The pull
// buffer must hold values that stream into it, so each entry B_j(z) takes the
// equilibrium of node z + c_j; where z + c_j lies beyond a wall, the link is
// the bounce-back one and B_j(z) holds the opposite direction's value at z.
// in = [phi0 | ux0 | uy0 | p0] as doubles (N each).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void eq_at(const double* __restrict__ in, size_t N, size_t s, int i,
                                      const Model& m, float& fe, float& ge) {
    const float phi = (float)in[s];
    const float ux = (float)in[N + s], uy = (float)in[2 * N + s], p = (float)in[3 * N + s];
    const float rho = fma_rn(phi, m.drho, m.rho_g);
    float cu[9];
    cdot9(ux, uy, cu);
    const float usq = fma_rn(ux, ux, mul(uy, uy));
    fe = feq_i(i, phi, cu[i]);
    ge = geq_i(i, mul(3.f, p), rho, cu[i], usq);
}

template <int ST>
__global__ void k_init(const double* __restrict__ in, void* __restrict__ fd,
                       void* __restrict__ gd, float* __restrict__ phiu, int nx, int ny, Model m) {
    const size_t N = (size_t)nx * ny;
    const int N32 = (int)N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int yy = y + cy_of(j);
            float fe, ge;
            if (m.walls && (yy < 0 || yy >= ny)) {
                eq_at(in, N, n, opp_of(j), m, fe, ge);
            } else {
                const int xs = fold_x(x + cx_of(j), nx), ys = fold_y(yy, ny, 0);
                eq_at(in, N, (size_t)ys * nx + xs, j, m, fe, ge);
            }
            Pop<ST>::putf(fd, N32, j, (int)n, fe);
            Pop<ST>::putg(fd, gd, N32, j, (int)n, ge);
        }
        const float phi = (float)in[n];
        {
            // the node's own pulled f_j are its (stored) equilibria; f_0 takes
            // the remainder so the stored populations sum to phi0
            float d[9], fe, ge;
#pragma unroll
            for (int j = 1; j < 9; ++j) {
                eq_at(in, N, n, j, m, fe, ge);
                d[j] = fe;
            }
            Pop<ST>::putf(fd, N32, 0, (int)n, Pop<ST>::init_rest(phi, d));
        }
        phiu[n] = mul(phi, (float)in[N + n]);
        phiu[N + n] = mul(phi, (float)in[2 * N + n]);
    }
}

// Checkpoint out: canonical pre-collision state = the pulled populations.
template <int ST>
__global__ void k_state_out(const void* __restrict__ fs, const void* __restrict__ gs,
                            const float* __restrict__ phiu, float* __restrict__ st, int nx,
                            int ny, int walls) {
    const size_t N = (size_t)nx * ny;
    const int N32 = (int)N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
        const Nbr q = make_nbr(x, y, nx, ny, walls);
        float v[9], w[9];
        pull18<ST>(fs, gs, N32, q, v, w);
        Pop<ST>::canon(v, w);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            st[i * N + n] = v[i];
            st[(9 + i) * N + n] = w[i];
        }
        st[18 * N + n] = phiu[n];
        st[19 * N + n] = phiu[N + n];
    }
}

// Checkpoint in: the inverse permutation of the pull (see k_init).  With
// 16-bit storage the rest population takes the rounding of the node's moving
// ones, so the stored node sums equal the given ones (a saved state restores
// bit for bit: its moving populations are already representable).
template <int ST>
__global__ void k_state_in(const float* __restrict__ st, void* __restrict__ fd,
                           void* __restrict__ gd, float* __restrict__ phiu, int nx, int ny,
                           int walls) {
    const size_t N = (size_t)nx * ny;
    const int N32 = (int)N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
         n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int yy = y + cy_of(j);
            size_t src;
            int dir;
            if (walls && (yy < 0 || yy >= ny)) {
                src = n;
                dir = opp_of(j);
            } else {
                src = (size_t)fold_y(yy, ny, 0) * nx + fold_x(x + cx_of(j), nx);
                dir = j;
            }
            Pop<ST>::putf(fd, N32, j, (int)n, st[dir * N + src]);
            Pop<ST>::putg(fd, gd, N32, j, (int)n, st[(9 + dir) * N + src]);
        }
        {
            float c = st[n];
#pragma unroll
            for (int j = 1; j < 9; ++j) {
                const float v = st[j * N + n];
                c = add(c, sub(v, Pop<ST>::round_f(j, v)));
            }
            Pop<ST>::putf(fd, N32, 0, (int)n, c);
        }
        phiu[n] = st[18 * N + n];
        phiu[N + n] = st[19 * N + n];
    }
}

// Grid reductions over the fields buffer [phi|rho|ux|uy|p] (doubles):
// block partials (sum phi, max |u|, min p, max p) into scratch, then one block
// folds the partials in a fixed order.
constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS)
    k_diag_partial(const double* __restrict__ fields, size_t N, double* __restrict__ part) {
    __shared__ double s_sum[RED_THREADS], s_um[RED_THREADS], s_pmin[RED_THREADS],
        s_pmax[RED_THREADS];
    double sum = 0.0, um = 0.0, pmin = INFINITY, pmax = -INFINITY;
    for (size_t n = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; n < N;
         n += (size_t)gridDim.x * RED_THREADS) {
        sum += fields[n];
        const double ux = fields[2 * N + n], uy = fields[3 * N + n], p = fields[4 * N + n];
        um = fmax(um, sqrt(ux * ux + uy * uy));
        pmin = fmin(pmin, p);
        pmax = fmax(pmax, p);
    }
    const int t = threadIdx.x;
    s_sum[t] = sum;
    s_um[t] = um;
    s_pmin[t] = pmin;
    s_pmax[t] = pmax;
    __syncthreads();
    for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
        if (t < h) {
            s_sum[t] += s_sum[t + h];
            s_um[t] = fmax(s_um[t], s_um[t + h]);
            s_pmin[t] = fmin(s_pmin[t], s_pmin[t + h]);
            s_pmax[t] = fmax(s_pmax[t], s_pmax[t + h]);
        }
        __syncthreads();
    }
    if (t == 0) {
        part[4 * blockIdx.x + 0] = s_sum[0];
        part[4 * blockIdx.x + 1] = s_um[0];
        part[4 * blockIdx.x + 2] = s_pmin[0];
        part[4 * blockIdx.x + 3] = s_pmax[0];
    }
}

__global__ void __launch_bounds__(RED_THREADS)
    k_diag_final(const double* __restrict__ part, int nb, double* __restrict__ res) {
    __shared__ double s_sum[RED_THREADS], s_um[RED_THREADS], s_pmin[RED_THREADS],
        s_pmax[RED_THREADS];
    const int t = threadIdx.x;
    double sum = 0.0, um = 0.0, pmin = INFINITY, pmax = -INFINITY;
    for (int b = t; b < nb; b += RED_THREADS) {
        sum += part[4 * b];
        um = fmax(um, part[4 * b + 1]);
        pmin = fmin(pmin, part[4 * b + 2]);
        pmax = fmax(pmax, part[4 * b + 3]);
    }
    s_sum[t] = sum;
    s_um[t] = um;
    s_pmin[t] = pmin;
    s_pmax[t] = pmax;
    __syncthreads();
    for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
        if (t < h) {
            s_sum[t] += s_sum[t + h];
            s_um[t] = fmax(s_um[t], s_um[t + h]);
            s_pmin[t] = fmin(s_pmin[t], s_pmin[t + h]);
            s_pmax[t] = fmax(s_pmax[t], s_pmax[t + h]);
        }
        __syncthreads();
    }
    if (t == 0) {
        res[0] = s_sum[0];
        res[1] = s_um[0];
        res[2] = s_pmin[0];
        res[3] = s_pmax[0];
    }
}

// direct-load step: TX x TY threads, one node each (overridable at build time)
constexpr int STEP_TX = LBM_STEP_TX;
// thread-block width of the 16-bit steps
#ifndef LBM_STEP16_TX
#define LBM_STEP16_TX 32
#endif
constexpr int STEP16_TX = LBM_STEP16_TX;
constexpr int STEP_TY = LBM_STEP_TY;
constexpr int RED_BLOCKS = 1216;  // 8 x 152 SMs
}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct lbm_handle {
    int nx = 0, ny = 0;
    size_t N = 0;
    int device = 0;
    lbm_params prm{};
    Model model{};
    cudaStream_t stream = nullptr;
    float* f[2] = {nullptr, nullptr};
    float* g[2] = {nullptr, nullptr};
    float* phiu = nullptr;
    int cur = 0;
    void* staging = nullptr;   // host I/O staging: max(5 N doubles, 20 N floats)
    double* red_part = nullptr;  // RED_BLOCKS x 4 partials
    double* red_res = nullptr;   // 4 results
    unsigned int* flag = nullptr;
    bool inited = false;
    long long since_check = 0;
    int pf_ahead = 0;  // L2 prefetch distance of the step kernel, in tiles
    bool owns_memory = true;  // false: the device buffers live in a caller's workspace
    unsigned long long nstep = 0;  // steps since lbm_init: seeds the stochastic rounding
    PfMaps pm[2] = {};             // prefetch tensor maps of the step reading buffer 0 / 1
    char err[512] = {0};
};

static lbm_status fail(lbm_handle* h, lbm_status st, const char* fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof h->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

#define LBM_CUDA(h, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(h, LBM_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                        __FILE__, __LINE__);                                                \
    } while (0)

static lbm_status validate(int nx, int ny, const lbm_params* p, char* msg, size_t len) {
    auto bad = [&](const char* why) {
        snprintf(msg, len, "invalid parameters: %s", why);
        return LBM_ERR_INVALID;
    };
    if (!p) return bad("params is NULL");
    if (nx < 1 || ny < 1) return bad("nx and ny must be >= 1");
    if ((long long)nx * ny >= (1LL << 31) / 20) return bad("grid too large (nx*ny*20 must fit in 2^31)");
    if (!(p->rho_l > 0) || !(p->rho_g > 0)) return bad("rho_l and rho_g must be > 0");
    if (!(p->nu_l > 0) || !(p->nu_g > 0)) return bad("nu_l and nu_g must be > 0");
    if (p->visc_mode < 0 || p->visc_mode > 2) return bad("visc_mode must be 0, 1 or 2");
    if (!(p->sigma >= 0)) return bad("sigma must be >= 0");
    if (!(p->W > 0)) return bad("W must be > 0");
    if (!(p->tau_h > 0.5)) return bad("tau_h must be > 0.5");
    if (!std::isfinite(p->Gx) || !std::isfinite(p->Gy)) return bad("G must be finite");
    if (p->bc_y != LBM_BC_PERIODIC && p->bc_y != LBM_BC_WALLS && p->bc_y != LBM_BC_WALL_OPEN)
        return bad("bc_y must be LBM_BC_PERIODIC, LBM_BC_WALLS or LBM_BC_WALL_OPEN");
    if (p->bc_y == LBM_BC_WALL_OPEN && ny < 2)
        return bad("LBM_BC_WALL_OPEN needs ny >= 2 (the open top repeats the row below)");
    if (p->normal_scheme != LBM_NORMAL_CENTRAL && p->normal_scheme != LBM_NORMAL_LOCAL)
        return bad("normal_scheme must be 0 or 1");
    if (p->storage != LBM_STORE_FP32 && p->storage != LBM_STORE_FP16_SHIFTED &&
        p->storage != LBM_STORE_BF16_SHIFTED && p->storage != LBM_STORE_BF16_SHIFTED_SR)
        return bad("storage must be LBM_STORE_FP32, _FP16_SHIFTED, _BF16_SHIFTED or _BF16_SHIFTED_SR");
    if (p->check_every < 0) return bad("check_every must be >= 0");
    if (p->kernel != LBM_KERNEL_AUTO && p->kernel != LBM_KERNEL_GENERIC)
        return bad("kernel must be LBM_KERNEL_AUTO or LBM_KERNEL_GENERIC");
    return LBM_OK;
}

static Model make_model(const lbm_params& p) {
    Model m{};
    m.rho_g = (float)p.rho_g;
    m.drho = (float)(p.rho_l - p.rho_g);
    m.beta4 = (float)(4.0 * 12.0 * p.sigma / p.W);
    m.kappa = (float)(1.5 * p.sigma * p.W);
    m.Gx = (float)p.Gx;
    m.Gy = (float)p.Gy;
    m.inv_tau_f = (float)(1.0 / p.tau_h);
    m.tau_f_mh = (float)(p.tau_h - 0.5);
    m.four_over_W = (float)(4.0 / p.W);
    m.nu_l = (float)p.nu_l;
    m.nu_g = (float)p.nu_g;
    m.inv_nu_l = (float)(1.0 / p.nu_l);
    m.inv_nu_g = (float)(1.0 / p.nu_g);
    m.mu_l = (float)(p.rho_l * p.nu_l);
    m.mu_g = (float)(p.rho_g * p.nu_g);
    m.visc_mode = p.visc_mode;
    m.walls = p.bc_y;  // 0 periodic, 1 walls, 2 wall and open top
    m.local_normal = p.normal_scheme == LBM_NORMAL_LOCAL;
    m.check_nonfinite = p.check_every > 0;
    return m;
}

// The handle's own buffers are stream-ordered allocations on its stream
// (cudaMallocAsync / cudaFreeAsync), so creating and destroying handles does
// not synchronise the whole device.
static void release(lbm_handle* h) {
    if (!h->owns_memory) return;  // a caller's workspace stays the caller's
    void* bufs[9] = {h->f[0], h->f[1], h->g[0], h->g[1], h->phiu, h->staging, h->red_part,
                     h->red_res, h->flag};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, h->stream);
    cudaStreamSynchronize(h->stream);
}

// BF16_SHIFTED_SR stores the BF16 layout: initialisation, read-back,
// checkpoints and the impact tools use BF16's kernels
static bool is_bf16(int storage) {
    return storage == LBM_STORE_BF16_SHIFTED || storage == LBM_STORE_BF16_SHIFTED_SR;
}

static size_t f_bytes(int storage, size_t N) {
    return storage == LBM_STORE_FP32 ? Pop<ST_FP32>::f_bytes(N) : Pop<ST_FP16>::f_bytes(N);
}
static size_t g_bytes(int storage, size_t N) {
    return storage == LBM_STORE_FP32 ? Pop<ST_FP32>::g_bytes(N) : Pop<ST_FP16>::g_bytes(N);
}

// The device buffers of one handle, in workspace order, each starting on a
// 256-byte boundary: f[0], f[1], g[0], g[1], phi u, staging, block partials,
// results, flag.
struct Layout {
    size_t size[9];
    size_t offset[9];
    size_t total;
};
static Layout layout_of(int nx, int ny, int storage) {
    const size_t N = (size_t)nx * ny;
    const size_t fpop = f_bytes(storage, N), gpop = g_bytes(storage, N);
    const size_t staging = (20 * N * sizeof(float) > 5 * N * sizeof(double)) ? 20 * N * sizeof(float)
                                                                              : 5 * N * sizeof(double);
    Layout L{{fpop, fpop, gpop, gpop, 2 * N * sizeof(float), staging, 4 * RED_BLOCKS * sizeof(double),
              4 * sizeof(double), sizeof(unsigned int)},
             {},
             0};
    size_t at = 0;
    for (int k = 0; k < 9; ++k) {
        L.offset[k] = at;
        at += (L.size[k] + 255) / 256 * 256;
    }
    L.total = at;
    return L;
}

static int grid1d(size_t N) {
    size_t b = (N + 255) / 256;
    return (int)(b < 4096 ? (b ? b : 1) : 4096);
}

// Step launches use programmatic dependent launch (griddep_wait in the
// kernels): the next step's CTAs are scheduled while the previous step's
// last wave finishes, instead of after it.
#ifndef LBM_PDL
#define LBM_PDL 1
#endif
template <typename... Exp, typename... Act>
static cudaError_t launch_dep(void (*k)(Exp...), dim3 grid, dim3 block, cudaStream_t s, Act&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = LBM_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Act>(args)...);
}

static lbm_status launch_step(lbm_handle* h, bool fields, double* out) {
    const int c = h->cur;
    const bool walls = h->model.walls != 0;
    // a 16-bit step's thread takes LBM_NPT16 nodes, so its tile is that many times taller
    const bool st16 = !fields && h->prm.storage != LBM_STORE_FP32;
    const int tw = st16 ? STEP16_TX : STEP_TX;
    const int th = st16 ? STEP_TY * LBM_NPT16 : STEP_TY;
    dim3 block(tw, STEP_TY);
    dim3 grid((h->nx + tw - 1) / tw, (h->ny + th - 1) / th);
    using K = void (*)(const float*, const float*, float*, float*, float*, unsigned int*, double*,
                       int, int, Model, int, int, PfMaps);
    K k;
    // the steps of a handle that asked for non-finite checks test every node;
    // the others are compiled without the test (2% of the 16-bit step)
    const bool chk = h->model.check_nonfinite != 0;
#define LBM_STEP_KERNEL(ST_, TW_)                                                                 \
    (fields ? k_step<STEP_TX, STEP_TY, true, -1, ST_>                                            \
            : (walls ? (chk ? k_step<TW_, STEP_TY, false, 1, ST_, true>                          \
                            : k_step<TW_, STEP_TY, false, 1, ST_, false>)                        \
                     : (chk ? k_step<TW_, STEP_TY, false, 0, ST_, true>                          \
                            : k_step<TW_, STEP_TY, false, 0, ST_, false>)))
    switch (h->prm.storage) {
        case LBM_STORE_FP16_SHIFTED: k = LBM_STEP_KERNEL(ST_FP16, STEP16_TX); break;
        case LBM_STORE_BF16_SHIFTED: k = LBM_STEP_KERNEL(ST_BF16, STEP16_TX); break;
        // the read-back of the stochastically rounded format is BF16's
        case LBM_STORE_BF16_SHIFTED_SR:
            k = fields ? LBM_STEP_KERNEL(ST_BF16, STEP16_TX) : LBM_STEP_KERNEL(ST_BF16_SR, STEP16_TX);
            break;
        default: k = LBM_STEP_KERNEL(ST_FP32, STEP_TX);
    }
#undef LBM_STEP_KERNEL
    if (fields)
        k<<<grid, block, 0, h->stream>>>(h->f[c], h->g[c], nullptr, nullptr, h->phiu, h->flag, out,
                                         h->nx, h->ny, h->model, 0, 0, PfMaps{});
    else {
        // a distinct seed per step (the golden-ratio multiple of the step count)
        h->model.seed = (unsigned int)(++h->nstep) * 0x9e3779b9u;
        LBM_CUDA(h, launch_dep(k, grid, block, h->stream, (const float*)h->f[c],
                               (const float*)h->g[c], h->f[c ^ 1], h->g[c ^ 1], h->phiu, h->flag,
                               (double*)nullptr, h->nx, h->ny, h->model, h->pf_ahead,
                               LBM_ALTERNATE_ORDER ? c : 0, h->pm[c]));
    }
    LBM_CUDA(h, cudaGetLastError());
    if (!fields) h->cur ^= 1;
    return LBM_OK;
}

static lbm_status check_flag(lbm_handle* h) {
    unsigned int v = 0;
    LBM_CUDA(h, cudaMemcpyAsync(&v, h->flag, sizeof v, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->since_check = 0;
    if (v) {
        LBM_CUDA(h, cudaMemsetAsync(h->flag, 0, sizeof(unsigned int), h->stream));
        if (v & 2u)
            return fail(h, LBM_ERR_CUDA, "a bulk tensor copy did not complete within the wait limit");
        if (v & 4u)
            return fail(h, LBM_ERR_CUDA, "an index check of the debug build failed");
        return fail(h, LBM_ERR_NONFINITE, "non-finite phi, u or p produced by a step");
    }
    return LBM_OK;
}

extern "C" {

// Shared by lbm_create (ws == NULL: the handle allocates its buffers) and
// lbm_create_in (the buffers are carved from the caller's workspace ws).
// Tensor maps of the step's L2 prefetch (PfMaps), for the step reading each
// population buffer: the planes of one set as one 3-D tensor (x, y, plane),
// the 16-bit f_0 and g_0 planes as 2-D tensors, and the two (phi u) planes;
// the box is one tile wide and its rows plus the two halo rows high.  Built
// only when a tiled tensor map's rules hold (row pitch a multiple of 16 bytes:
// nx % 8 == 0 covers the 2-byte g_0 plane; plane pitch likewise; the box
// inside the grid); otherwise, or if the driver lacks the encoder, the step
// keeps its per-thread prefetch requests.
// cuTensorMapEncodeTiled of the driver, or nullptr
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            enc = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    return enc;
}

// A prefetch map over `planes` planes of nx x ny elements of es bytes at
// base (one plane: a 2-D map), with a box of bx x by elements and every plane.
// The caller guarantees nx % 8 == 0 (row and plane pitches multiples of 16
// bytes) and a 16-byte aligned base.
static bool encode_prefetch_map(CUtensorMap* m, CUtensorMapDataType t, int es, void* base,
                                int planes, int nx, int ny, int bx, int by) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t N = (cuuint64_t)nx * ny;
    const cuuint32_t rank = planes > 1 ? 3 : 2;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * es, N * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, t, rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The four 16-bit prefetch maps of buffer c of handle h (word planes, f_0,
// g_0, (phi u)), box bx x by
static bool encode_maps16(const lbm_handle* h, int c, CUtensorMap m[4], int bx, int by) {
    const int nx = h->nx, ny = h->ny;
    const size_t N = h->N;
    return encode_prefetch_map(&m[0], CU_TENSOR_MAP_DATA_TYPE_UINT32, 4,
                               static_cast<char*>((void*)h->f[c]) + 4 * N, 8, nx, ny, bx, by) &&
           encode_prefetch_map(&m[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->f[c], 1, nx, ny, bx, by) &&
           encode_prefetch_map(&m[2], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, h->g[c], 1, nx, ny, bx, by) &&
           encode_prefetch_map(&m[3], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->phiu, 2, nx, ny, bx, by);
}

static void encode_pf_maps(lbm_handle* h) {
    h->pm[0].on = h->pm[1].on = 0;
    if (!LBM_TMA_PREFETCH) return;
    if (h->prm.storage == LBM_STORE_FP32 && !LBM_TMA_PREFETCH32) return;
    const bool st16 = h->prm.storage != LBM_STORE_FP32;
    const int tx = st16 ? STEP16_TX : STEP_TX;
    const int th = st16 ? STEP_TY * LBM_NPT16 : STEP_TY;
    const int nx = h->nx, ny = h->ny;
    if (nx % 8 != 0 || nx < tx || ny < th + 2) return;
    for (int c = 0; c < 2; ++c) {
        PfMaps& pm = h->pm[c];
        bool ok;
        if (st16) {
            CUtensorMap m[4];
            ok = encode_maps16(h, c, m, tx, th + 2);
            if (ok) {
                pm.pop[0] = m[0];
                pm.pop[1] = m[1];
                pm.pop[2] = m[2];
                pm.phiu = m[3];
            }
        } else {
            ok = encode_prefetch_map(&pm.pop[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->f[c], 9, nx, ny,
                                     tx, th + 2) &&
                 encode_prefetch_map(&pm.pop[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->g[c], 9, nx, ny,
                                     tx, th + 2) &&
                 encode_prefetch_map(&pm.phiu, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->phiu, 2, nx, ny,
                                     tx, th + 2);
        }
        if (!ok) {
            h->pm[0].on = h->pm[1].on = 0;
            return;
        }
        pm.on = 1;
    }
}

static lbm_status create_handle(int nx, int ny, const lbm_params* p, void* ws, lbm_handle** out) {
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ERR_OOM;
    h->nx = nx;
    h->ny = ny;
    h->N = (size_t)nx * ny;
    h->prm = *p;
    h->model = make_model(*p);
    h->stream = (cudaStream_t)p->stream;
    h->owns_memory = ws == nullptr;
    cudaError_t e = cudaGetDevice(&h->device);
    const Layout L = layout_of(nx, ny, p->storage);
    void** slot[9] = {(void**)&h->f[0], (void**)&h->f[1], (void**)&h->g[0], (void**)&h->g[1],
                      (void**)&h->phiu, &h->staging,      (void**)&h->red_part, (void**)&h->red_res,
                      (void**)&h->flag};
    for (int k = 0; k < 9 && e == cudaSuccess; ++k) {
        if (ws)
            *slot[k] = static_cast<char*>(ws) + L.offset[k];
        else
            e = cudaMallocAsync(slot[k], L.size[k], h->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flag, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const bool st16 = p->storage != LBM_STORE_FP32;
    h->pf_ahead = (st16 ? (p->bc_y != LBM_BC_PERIODIC ? LBM_PREFETCH16_WALLS_PER10SM : LBM_PREFETCH16_PER10SM)
                        : LBM_PREFETCH_PER10SM) * sms / 10;
    {
        // The prefetch pays only when a step's traffic does not fit in L2:
        // below, the rows it asks for are mostly there already and the requests
        // only cost issue slots (measured: FP16 on the 2400 x 600 impact, 132 MB
        // per step against a 129 MB L2, 48.7 k MLUPS without and 43.7 k with).
        int l2 = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device);
        const double bytes = (st16 ? 92.0 : 160.0) * (double)nx * ny;
        const bool maps16 = st16 && LBM_TMA_PREFETCH && nx % 8 == 0;  // tensor maps likely
        const int thr = !st16 ? LBM_PREFETCH_L2X10 : maps16 ? LBM_PREFETCH16_TMA_L2X10 : LBM_PREFETCH16_L2X10;
        if (bytes * 10.0 < (double)thr * l2) h->pf_ahead = 0;
        if (e == cudaSuccess && h->pf_ahead > 0) {
            encode_pf_maps(h);
            // no maps after all: the per-thread requests' own threshold
            if (st16 && !h->pm[0].on && bytes * 10.0 < (double)LBM_PREFETCH16_L2X10 * l2) h->pf_ahead = 0;
        }
    }
    if (e != cudaSuccess) {
        fprintf(stderr, "lbm_create: %s\n", cudaGetErrorString(e));
        release(h);
        delete h;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_create(int nx, int ny, const lbm_params* p, lbm_handle** out) {
    if (!out) return LBM_ERR_INVALID;
    *out = nullptr;
    char msg[256];
    lbm_status st = validate(nx, ny, p, msg, sizeof msg);
    if (st != LBM_OK) {
        fprintf(stderr, "lbm_create: %s\n", msg);
        return st;
    }
    return create_handle(nx, ny, p, nullptr, out);
}

lbm_status lbm_workspace_bytes(int nx, int ny, const lbm_params* p, size_t* bytes) {
    if (!bytes) return LBM_ERR_INVALID;
    *bytes = 0;
    char msg[256];
    lbm_status st = validate(nx, ny, p, msg, sizeof msg);
    if (st != LBM_OK) {
        fprintf(stderr, "lbm_workspace_bytes: %s\n", msg);
        return st;
    }
    *bytes = layout_of(nx, ny, p->storage).total;
    return LBM_OK;
}

lbm_status lbm_create_in(int nx, int ny, const lbm_params* p, void* d_workspace, size_t bytes,
                         lbm_handle** out) {
    if (!out) return LBM_ERR_INVALID;
    *out = nullptr;
    char msg[256];
    lbm_status st = validate(nx, ny, p, msg, sizeof msg);
    if (st != LBM_OK) {
        fprintf(stderr, "lbm_create_in: %s\n", msg);
        return st;
    }
    const size_t need = layout_of(nx, ny, p->storage).total;
    if (!d_workspace || bytes < need || ((uintptr_t)d_workspace % 256) != 0) {
        fprintf(stderr, "lbm_create_in: need a 256-byte aligned device workspace of at least %zu "
                        "bytes, got %p and %zu bytes\n", need, d_workspace, bytes);
        return LBM_ERR_INVALID;
    }
    // the workspace must be device (or managed) memory of the current device:
    // a host pointer here would make every kernel fault
    cudaPointerAttributes at{};
    int dev = -1;
    if (cudaPointerGetAttributes(&at, d_workspace) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
        cudaGetLastError();
        fprintf(stderr, "lbm_create_in: the workspace is not device memory of the current device\n");
        return LBM_ERR_INVALID;
    }
    return create_handle(nx, ny, p, d_workspace, out);
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err : "null handle"; }

size_t lbm_state_bytes(const lbm_handle* h) { return h ? 20 * h->N * sizeof(float) : 0; }

lbm_status lbm_init(lbm_handle* h, const double* phi0, const double* ux0, const double* uy0,
                    const double* p0) {
    if (!h) return LBM_ERR_INVALID;
    if (!phi0) return fail(h, LBM_ERR_INVALID, "lbm_init: phi0 is NULL");
    LBM_CUDA(h, cudaSetDevice(h->device));
    double* in = (double*)h->staging;
    const size_t bytes = h->N * sizeof(double);
    const double* src[4] = {phi0, ux0, uy0, p0};
    for (int k = 0; k < 4; ++k) {
        if (src[k])
            LBM_CUDA(h, cudaMemcpyAsync(in + k * h->N, src[k], bytes, cudaMemcpyHostToDevice,
                                        h->stream));
        else
            LBM_CUDA(h, cudaMemsetAsync(in + k * h->N, 0, bytes, h->stream));
    }
    h->cur = 0;
    auto kinit = h->prm.storage == LBM_STORE_FP16_SHIFTED ? k_init<ST_FP16>
                 : is_bf16(h->prm.storage)                ? k_init<ST_BF16>
                                                          : k_init<ST_FP32>;
    kinit<<<grid1d(h->N), 256, 0, h->stream>>>(in, h->f[0], h->g[0], h->phiu, h->nx, h->ny,
                                                 h->model);
    LBM_CUDA(h, cudaGetLastError());
    LBM_CUDA(h, cudaMemsetAsync(h->flag, 0, sizeof(unsigned int), h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->inited = true;
    h->nstep = 0;
    h->since_check = 0;
    return LBM_OK;
}

lbm_status lbm_step(lbm_handle* h, int nsteps) {
    if (!h) return LBM_ERR_INVALID;
    if (nsteps < 0) return fail(h, LBM_ERR_INVALID, "lbm_step: nsteps < 0");
    if (!h->inited) return fail(h, LBM_ERR_STATE, "lbm_step before lbm_init");
    LBM_CUDA(h, cudaSetDevice(h->device));
    for (int s = 0; s < nsteps; ++s) {
        lbm_status st = launch_step(h, false, nullptr);
        if (st != LBM_OK) return st;
        if (h->prm.check_every > 0 && ++h->since_check >= h->prm.check_every) {
            st = check_flag(h);
            if (st != LBM_OK) return st;
        }
    }
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_handle* h, double* phi, double* rho, double* ux, double* uy,
                          double* p) {
    if (!h) return LBM_ERR_INVALID;
    if (!h->inited) return fail(h, LBM_ERR_STATE, "lbm_get_fields before lbm_init");
    LBM_CUDA(h, cudaSetDevice(h->device));
    double* buf = (double*)h->staging;
    lbm_status st = launch_step(h, true, buf);
    if (st != LBM_OK) return st;
    double* outs[5] = {phi, rho, ux, uy, p};
    for (int k = 0; k < 5; ++k)
        if (outs[k])
            LBM_CUDA(h, cudaMemcpyAsync(outs[k], buf + k * h->N, h->N * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_handle* h, void* host_buf, size_t bytes) {
    if (!h || !host_buf) return fail(h, LBM_ERR_INVALID, "lbm_get_state: NULL argument");
    if (bytes != lbm_state_bytes(h))
        return fail(h, LBM_ERR_INVALID, "lbm_get_state: need %zu bytes, got %zu",
                    lbm_state_bytes(h), bytes);
    if (!h->inited) return fail(h, LBM_ERR_STATE, "lbm_get_state before lbm_init");
    LBM_CUDA(h, cudaSetDevice(h->device));
    float* st = (float*)h->staging;
    auto kout = h->prm.storage == LBM_STORE_FP16_SHIFTED ? k_state_out<ST_FP16>
                : is_bf16(h->prm.storage)                ? k_state_out<ST_BF16>
                                                          : k_state_out<ST_FP32>;
    kout<<<grid1d(h->N), 256, 0, h->stream>>>(h->f[h->cur], h->g[h->cur], h->phiu, st,
                                                      h->nx, h->ny, h->model.walls);
    LBM_CUDA(h, cudaGetLastError());
    LBM_CUDA(h, cudaMemcpyAsync(host_buf, st, bytes, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_handle* h, const void* host_buf, size_t bytes) {
    if (!h || !host_buf) return fail(h, LBM_ERR_INVALID, "lbm_set_state: NULL argument");
    if (bytes != lbm_state_bytes(h))
        return fail(h, LBM_ERR_INVALID, "lbm_set_state: need %zu bytes, got %zu",
                    lbm_state_bytes(h), bytes);
    LBM_CUDA(h, cudaSetDevice(h->device));
    float* st = (float*)h->staging;
    LBM_CUDA(h, cudaMemcpyAsync(st, host_buf, bytes, cudaMemcpyHostToDevice, h->stream));
    h->cur = 0;
    auto kin = h->prm.storage == LBM_STORE_FP16_SHIFTED ? k_state_in<ST_FP16>
               : is_bf16(h->prm.storage)                ? k_state_in<ST_BF16>
                                                         : k_state_in<ST_FP32>;
    kin<<<grid1d(h->N), 256, 0, h->stream>>>(st, h->f[0], h->g[0], h->phiu, h->nx,
                                                     h->ny, h->model.walls);
    LBM_CUDA(h, cudaGetLastError());
    LBM_CUDA(h, cudaMemsetAsync(h->flag, 0, sizeof(unsigned int), h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->inited = true;
    h->since_check = 0;
    return LBM_OK;
}

lbm_status lbm_diag(lbm_handle* h, double* sum_phi, double* umax, double* pmin, double* pmax) {
    if (!h) return LBM_ERR_INVALID;
    if (!h->inited) return fail(h, LBM_ERR_STATE, "lbm_diag before lbm_init");
    LBM_CUDA(h, cudaSetDevice(h->device));
    double* buf = (double*)h->staging;
    lbm_status st = launch_step(h, true, buf);
    if (st != LBM_OK) return st;
    k_diag_partial<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(buf, h->N, h->red_part);
    LBM_CUDA(h, cudaGetLastError());
    k_diag_final<<<1, RED_THREADS, 0, h->stream>>>(h->red_part, RED_BLOCKS, h->red_res);
    LBM_CUDA(h, cudaGetLastError());
    double r[4];
    LBM_CUDA(h, cudaMemcpyAsync(r, h->red_res, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (sum_phi) *sum_phi = r[0];
    if (umax) *umax = r[1];
    if (pmin) *pmin = r[2];
    if (pmax) *pmax = r[3];
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_handle* h) {
    if (!h) return LBM_ERR_INVALID;
    LBM_CUDA(h, cudaSetDevice(h->device));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free grid reduction.
//
// Some callers may not allocate device memory at the point where they want
// diagnostics: a host process whose device memory is handed out by its own
// pool or runtime (so a cudaMalloc behind its back would break its
// accounting or fail outright), or a time-stepping loop that must not
// synchronise the device, which cudaMalloc and cudaFree can do.
// lbm_diag_fields_noalloc serves them: it reduces fields the caller already
// holds on the device, with the block partials in the file-scope array below
// instead of the handle's cudaMalloc'd buffer.  The array is part of the
// library image, so every GPU that loads the library holds it (128 KiB) until
// the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_MAX_BLOCKS = 4096;       // partials the array can hold
constexpr size_t NOALLOC_PER_BLOCK = 4096;     // elements reduced per block
constexpr size_t NOALLOC_MAX_N = NOALLOC_MAX_BLOCKS * NOALLOC_PER_BLOCK;  // 16,777,216
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_part[4 * NOALLOC_MAX_BLOCKS];

// Host side: the array's name is only a host stand-in, never a device
// address.  Its device address is looked up per device, with that device
// current, and cached together with the identity of the context it was
// looked up in: after a device reset the primary context (and with it the
// library's module) is new, and the next call looks the address up again.
struct NoallocSlot {
    unsigned long long ctx_id = 0;  // 0: not set up
    void* ptr = nullptr;
};
static NoallocSlot g_noalloc_slot[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

static void noalloc_msg(char* err, size_t len, const char* fmt, ...) {
    if (!err || len == 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, len, fmt, ap);
    va_end(ap);
}

// Unique identity of the calling thread's current context (0 when none is
// current yet), through the driver entry points the runtime exposes, so the
// library needs no link against libcuda.
static cudaError_t current_context_id(unsigned long long* id) {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    *id = 0;
    if (!get_current || !get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000,
                                                         cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorSymbolNotFound;
        get_current = (PFN_cuCtxGetCurrent_v4000)f1;
        get_id = (PFN_cuCtxGetId_v12000)f2;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    if (!ctx) return cudaSuccess;
    if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_diag_fields_noalloc(const double* d_fields, size_t n, double* d_out,
                                              void* stream, char* err, size_t err_len) {
    if (err && err_len) err[0] = '\0';
    if (!d_fields && n > 0) {
        noalloc_msg(err, err_len, "lbm_diag_fields_noalloc: d_fields is NULL");
        return LBM_ERR_INVALID;
    }
    if (!d_out) {
        noalloc_msg(err, err_len, "lbm_diag_fields_noalloc: d_out is NULL");
        return LBM_ERR_INVALID;
    }
    if (n > NOALLOC_MAX_N) {
        noalloc_msg(err, err_len,
                    "lbm_diag_fields_noalloc: n = %zu exceeds the maximum of %zu nodes "
                    "(%d static partial slots x %zu nodes each)",
                    n, NOALLOC_MAX_N, NOALLOC_MAX_BLOCKS, NOALLOC_PER_BLOCK);
        return LBM_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        noalloc_msg(err, err_len, "lbm_diag_fields_noalloc: no usable current device (%s)",
                    cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    // an error left by earlier, unrelated work is reported as such and left
    // pending for its owner
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        noalloc_msg(err, err_len,
                    "lbm_diag_fields_noalloc: an earlier CUDA error is pending (%s); nothing launched",
                    cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        NoallocSlot& slot = g_noalloc_slot[dev];
        unsigned long long id = 0;
        e = current_context_id(&id);
        if (e == cudaSuccess && (id == 0 || id != slot.ctx_id || !slot.ptr)) {
            // set-up, on the first call on this device and after a device
            // reset: the array's device address in the current context, and
            // both kernels loaded now (under lazy module loading a first
            // launch would load them)
            void* ptr = nullptr;
            cudaFuncAttributes fa;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_part);
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_diag_partial);
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_diag_final);
            if (e == cudaSuccess) e = current_context_id(&id);
            if (e == cudaSuccess && (!ptr || id == 0)) e = cudaErrorInvalidSymbol;
            if (e == cudaSuccess) {
                slot.ctx_id = id;
                slot.ptr = ptr;
            } else {
                slot = NoallocSlot();
            }
        }
        part = (double*)slot.ptr;
    }
    if (e != cudaSuccess) {
        noalloc_msg(err, err_len, "lbm_diag_fields_noalloc: set-up of the static array failed: %s",
                    cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // every slot the final pass reads is rewritten by this call's first pass
    const int nb = (int)((n + NOALLOC_PER_BLOCK - 1) / NOALLOC_PER_BLOCK);
    if (nb > 0) k_diag_partial<<<nb, RED_THREADS, 0, s>>>(d_fields, n, part);
    k_diag_final<<<1, RED_THREADS, 0, s>>>(part, nb, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        noalloc_msg(err, err_len, "lbm_diag_fields_noalloc: launch failed: %s",
                    cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Batched step: many independent cases (different sizes and parameters, one
// storage format) advanced together.  One kernel launch covers a global list
// of 32 x TY tiles over all cases, one block per tile (a tile table maps the
// block to its case and tile); each tile runs the same step_tile body
// as the single-case kernel, so a case advanced in a batch gives the same bits
// as the case advanced alone.  Steps run as replays of a captured CUDA graph;
// the tile height is picked by timing the candidates on the batch's own first
// steps (all candidates give the same bits, so those steps count).
// ---------------------------------------------------------------------------
namespace {

struct CaseDesc {
    float* f[2];
    float* g[2];
    float* phiu;
    unsigned int* flag;
    int nx, ny;
    int cur;   // buffer holding the current state when the batch parity is 0
    int map0;  // first of the case's 8 prefetch maps in BatchTable::maps (4 per buffer)
    Model m;
};

// The whole case table travels as a kernel parameter (constant bank): the
// block-uniform case data then needs no registers of the tile body.
constexpr int BATCH_MAX_CASES = 200;
// the box of the batched 16-bit kernels' prefetch maps (x, rows)
constexpr int BATCH_PF_BOX_X = 32, BATCH_PF_BOX_Y = 10;
struct BatchTable {
    const CUtensorMap* maps;  // 16-bit prefetch maps in device memory (nullptr: per-thread requests)
    int ncases;
    int tiles_x[BATCH_MAX_CASES];
    int tile0[BATCH_MAX_CASES + 1];  // first tile of each case; tile0[ncases] = total
    CaseDesc c[BATCH_MAX_CASES];
};
static_assert(sizeof(BatchTable) <= 32000, "kernel parameters are limited to 32 KB");

// resident threads per SM the batch kernels are compiled for (sets the
// register budget): 1280 = 10 blocks of 32 x 4, 48 registers, no spills.  On
// the 64-case sweep (MLUPS, FP32 / FP16 / BF16): 1024 threads 36.1 / 45.0 /
// 44.3 k, 1152: 36.8 / 47.6 / 46.6 k, 1280: 37.8 / 49.0 / 47.8 k; from 1408
// the kernels spill.
#ifndef LBM_BATCH_THREADS
#define LBM_BATCH_THREADS 1280
#endif
// L2 prefetch distance of the batched kernels, in tiles per 10 SMs (0: off)
#ifndef LBM_BATCH_PF_PER10SM
#define LBM_BATCH_PF_PER10SM 20
#endif
// nodes per thread of the batched 16-bit kernels (their tiles are this many
// times taller than the thread block)
#ifndef LBM_NPT16_BATCH
#define LBM_NPT16_BATCH 2
#endif
// resident threads per SM the batched 16-bit kernels are compiled for: 1024 =
// 8 blocks of 32 x 4 threads, 64 registers (two nodes per thread)
#ifndef LBM_BATCH_THREADS16
#define LBM_BATCH_THREADS16 1024
#endif

// One time step of every case of one boundary class (WALLS = 0: periodic in
// y, 1: walls in y): block t runs tile t of the class's tile list, whose
// entry holds (case, tile row << 16 | tile column).
template <int TX, int TY, int ST, int WALLS, bool CHK>
__global__ void __launch_bounds__(TX* TY, (ST == ST_FP32 ? LBM_BATCH_THREADS : LBM_BATCH_THREADS16) /
                                              (TX * TY))
    k_step_batch(const __grid_constant__ BatchTable T, const int2* __restrict__ tiles, int parity,
                 int pf_ahead) {
    __shared__ float sphi[TY * (ST == ST_FP32 ? 1 : LBM_NPT16_BATCH) + 2][TX + 2];
    griddep_wait();
    griddep_launch();
    constexpr int TH = TY * (ST == ST_FP32 ? 1 : LBM_NPT16_BATCH);  // tile height in nodes
    // odd steps walk the tile list backwards, as the single-case step does
    const bool rev = LBM_ALTERNATE_ORDER && (parity & 1);
    const int slot = rev ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    // L2 prefetch of the tile pf_ahead entries later in the walk, as in the
    // single-case step (0: off)
    if (pf_ahead > 0 && blockIdx.x + pf_ahead < gridDim.x) {
        const int2 pe = __ldg(tiles + (rev ? slot - pf_ahead : slot + pf_ahead));
        const CaseDesc& pc = T.c[pe.x < T.ncases ? pe.x : 0];
        const int pcur = (pc.cur + parity) & 1;
        if (ST != ST_FP32 && T.maps != nullptr) {
            // through the case's tensor maps, boxes of 32 x 10 elements:
            // (TX / 32) x ceil((TH + 2) / 10) boxes per map, one box of one
            // map per thread (as in the single-case 16-bit step)
            constexpr int SX = TX / BATCH_PF_BOX_X;
            constexpr int SY = (TH + 2 + BATCH_PF_BOX_Y - 1) / BATCH_PF_BOX_Y;
            const int t = threadIdx.y * TX + threadIdx.x;
            if (t < 4 * SX * SY) {
                const int k = t & 3, sub = t >> 2;
                const int x = (pe.y & 0xffff) * TX + BATCH_PF_BOX_X * (sub % SX);
                const int r0 = (pe.y >> 16) * TH;
                const int y = (r0 > 0 ? r0 - 1 : 0) + BATCH_PF_BOX_Y * (sub / SX);
                const CUtensorMap* mp = T.maps + pc.map0 + 4 * pcur + k;
                if (k == 1 || k == 2)
                    tma_prefetch_2d(mp, x, y);
                else
                    tma_prefetch_3d(mp, x, y, 0);
            }
        } else {
            prefetch_tile<TX, TH, TX * TY, ST>(pc.f[pcur], pc.g[pcur], pc.phiu, pc.nx, pc.ny, WALLS,
                                               pe.y & 0xffff, pe.y >> 16);
        }
    }
    const int2 e = __ldg(tiles + slot);
#if LBM_DEBUG_CHECKS
    if (e.x < 0 || e.x >= T.ncases || (e.y & 0xffff) * TX >= T.c[e.x < 0 || e.x >= T.ncases ? 0 : e.x].nx ||
        (e.y >> 16) * TY * (ST == ST_FP32 ? 1 : LBM_NPT16_BATCH) >=
            T.c[e.x < 0 || e.x >= T.ncases ? 0 : e.x].ny) {
        if (e.x >= 0 && e.x < T.ncases) atomicOr(T.c[e.x].flag, 4u);
        else atomicOr(T.c[0].flag, 4u);
        return;  // the whole block leaves before its barrier
    }
#endif
    const CaseDesc& cd = T.c[e.x];
    const int c = (cd.cur + parity) & 1;
    if constexpr (ST == ST_FP32) {
        step_tile<TX, TY, false, WALLS, ST, CHK>(sphi, cd.f[c], cd.g[c], cd.f[c ^ 1], cd.g[c ^ 1], cd.phiu,
                                            cd.flag, nullptr, cd.nx, cd.ny, cd.m, (e.y & 0xffff) * TX,
                                            (e.y >> 16) * TY);
    } else {
        step_tile16<TX, TY, LBM_NPT16_BATCH, WALLS, ST, CHK>(
            sphi, cd.f[c], cd.g[c], cd.f[c ^ 1], cd.g[c ^ 1], cd.phiu, cd.flag, cd.nx, cd.ny, cd.m,
            (e.y & 0xffff) * TX, (e.y >> 16) * TY * LBM_NPT16_BATCH);
    }
}

// boundary classes: each has its own specialised kernel, stream and tile shape
constexpr int BATCH_NCLASS = 2;  // 0: periodic cases, 1: walled cases
// tile shapes the tuner times (TX x TY nodes, one thread each)
constexpr int BATCH_NCAND = 5;
constexpr int BATCH_TX[BATCH_NCAND] = {32, 32, 32, 64, 64};
constexpr int BATCH_TY[BATCH_NCAND] = {4, 8, 16, 2, 4};
constexpr int BATCH_GRAPH_STEPS = 32;  // steps per graph replay (even)
// per shape: warm-up steps, then timed windows of steps; the shape's time is
// its fastest window (a single window let the choice between shapes within
// 2-3% of each other vary from run to run)
constexpr int BATCH_TUNE_WARM = 4, BATCH_TUNE_WINDOW = 12, BATCH_TUNE_WINDOWS = 2;
constexpr int BATCH_TUNE_PER_SHAPE = BATCH_TUNE_WARM + BATCH_TUNE_WINDOW * BATCH_TUNE_WINDOWS;

using BatchKernel = void (*)(BatchTable, const int2*, int, int);

// the batch kernels test for non-finite nodes when any case asked for checks
// (CHK), each case then by its own setting
template <int ST, int W, bool CHK>
BatchKernel batch_kernel(int cand) {
    switch (cand) {
        case 0: return k_step_batch<32, 4, ST, W, CHK>;
        case 2: return k_step_batch<32, 16, ST, W, CHK>;
        case 3: return k_step_batch<64, 2, ST, W, CHK>;
        case 4: return k_step_batch<64, 4, ST, W, CHK>;
        default: return k_step_batch<32, 8, ST, W, CHK>;
    }
}

template <int ST>
BatchKernel batch_kernel_st(int cls, int cand, bool chk) {
    if (chk) return cls ? batch_kernel<ST, 1, true>(cand) : batch_kernel<ST, 0, true>(cand);
    return cls ? batch_kernel<ST, 1, false>(cand) : batch_kernel<ST, 0, false>(cand);
}

BatchKernel batch_kernel_for(int storage, int cls, int cand, bool chk) {
    if (storage == LBM_STORE_FP16_SHIFTED) return batch_kernel_st<ST_FP16>(cls, cand, chk);
    if (storage == LBM_STORE_BF16_SHIFTED) return batch_kernel_st<ST_BF16>(cls, cand, chk);
    return batch_kernel_st<ST_FP32>(cls, cand, chk);
}

// Copy the non-finite flags of one class's cases to out[slot[j]] and clear
// them (one thread per case).
__global__ void k_batch_flags(const __grid_constant__ BatchTable T, const int* __restrict__ slot,
                              unsigned int* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= T.ncases) return;
    unsigned int* f = T.c[j].flag;
    out[slot[j]] = *f;
    *f = 0u;
}

}  // namespace

struct lbm_batch {
    int ncases = 0;
    std::vector<lbm_handle*> cases;
    std::vector<int> cls_of, slot_of;  // each case's class and its slot in the class table
    int ncls[BATCH_NCLASS] = {0, 0};
    int storage = 0;
    int device = 0;
    cudaStream_t user = nullptr;                 // the cases' stream
    cudaStream_t bs[BATCH_NCLASS] = {};          // private streams, one per class (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    BatchTable* table = nullptr;  // [class][shape], host side, passed by value
    int2* d_tiles[BATCH_NCLASS * BATCH_NCAND] = {};  // tile lists on the device, [class][shape]
    bool check = false;                 // some case asks for non-finite checks (check_every > 0)
    int* d_slot[BATCH_NCLASS] = {};     // per class: the batch index of each class slot
    unsigned int* d_flags = nullptr;    // gathered flags, one per case
    int cand[BATCH_NCLASS] = {1, 1};  // tile shape in use per class (index into BATCH_TX/TY)
    int pf_ahead = 0;                 // L2 prefetch distance in tiles (0: off)
    CUtensorMap* d_maps = nullptr;    // the 16-bit prefetch maps, 8 per case (nullptr: none)
    bool tuned = false;
    double tuned_us[BATCH_NCLASS][BATCH_NCAND] = {};
    cudaGraphExec_t graph = nullptr;
    bool failed = false;  // a step call failed after enqueueing work (see batch_abort)
    long long node_count = 0;
    char err[512] = {0};
    BatchTable& tab(int cls, int k) { return table[cls * BATCH_NCAND + k]; }
};

static lbm_status bfail(lbm_batch* b, lbm_status st, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof b->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

#define LBM_BCUDA(b, call)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail(b, LBM_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                         __FILE__, __LINE__);                                               \
    } while (0)

static void batch_release(lbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    delete[] b->table;
    for (int2* t : b->d_tiles)
        if (t) cudaFree(t);
    for (int* t : b->d_slot)
        if (t) cudaFree(t);
    if (b->d_flags) cudaFree(b->d_flags);
    if (b->d_maps) cudaFree(b->d_maps);
    for (cudaEvent_t e : {b->ev_in, b->ev_out, b->ev_fork, b->ev_join, b->t0, b->t1})
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < BATCH_NCLASS; ++k)
        if (b->bs[k]) cudaStreamDestroy(b->bs[k]);
}

// Take each case's current buffer from its handle (a case may have been
// stepped on its own since the last batch step); a change invalidates the
// captured graph, whose launches carry the tables.
static void batch_sync_table(lbm_batch* b) {
    bool changed = false;
    for (int c = 0; c < b->ncases; ++c)
        for (int k = 0; k < BATCH_NCAND; ++k) {
            CaseDesc& d = b->tab(b->cls_of[c], k).c[b->slot_of[c]];
            if (d.cur != b->cases[c]->cur) {
                d.cur = b->cases[c]->cur;
                changed = true;
            }
        }
    if (changed && b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// one step of class cls with tile shape cand, on the class's stream
static lbm_status batch_launch(lbm_batch* b, int cls, int cand, int parity) {
    BatchKernel k = batch_kernel_for(b->storage, cls, cand, b->check);
    const BatchTable& T = b->tab(cls, cand);
    // programmatic dependent launch, as for the single-case steps (also inside
    // the captured graph, where it becomes a programmatic edge)
    LBM_BCUDA(b, launch_dep(k, dim3(T.tile0[T.ncases]), dim3(BATCH_TX[cand], BATCH_TY[cand]),
                            b->bs[cls], T, (const int2*)b->d_tiles[cls * BATCH_NCAND + cand], parity,
                            b->pf_ahead));
    return LBM_OK;
}

// steps [from, to) of every non-empty class, each class on its own stream
static lbm_status batch_run(lbm_batch* b, long long from, long long to) {
    lbm_status st;
    for (int cls = 0; cls < BATCH_NCLASS; ++cls)
        if (b->ncls[cls])
            for (long long s = from; s < to; ++s)
                if ((st = batch_launch(b, cls, b->cand[cls], (int)(s & 1))) != LBM_OK) return st;
    return LBM_OK;
}

// the class streams start after, and end before, the work on bs[0]
static lbm_status batch_fork(lbm_batch* b) {
    LBM_BCUDA(b, cudaEventRecord(b->ev_fork, b->bs[0]));
    LBM_BCUDA(b, cudaStreamWaitEvent(b->bs[1], b->ev_fork, 0));
    return LBM_OK;
}
static lbm_status batch_join(lbm_batch* b) {
    LBM_BCUDA(b, cudaEventRecord(b->ev_join, b->bs[1]));
    LBM_BCUDA(b, cudaStreamWaitEvent(b->bs[0], b->ev_join, 0));
    return LBM_OK;
}

// A failure after the class streams forked: some steps of this call may be
// enqueued, so the cases' current buffers are unknown.  Join the class
// streams, order the cases' stream after them, and mark the batch and its
// cases as failed: each case needs lbm_init or lbm_set_state before further
// use, and the batch rejects further steps.
static lbm_status batch_abort(lbm_batch* b, lbm_status st) {
    cudaEventRecord(b->ev_join, b->bs[1]);
    cudaStreamWaitEvent(b->bs[0], b->ev_join, 0);
    cudaEventRecord(b->ev_out, b->bs[0]);
    cudaStreamWaitEvent(b->user, b->ev_out, 0);
    for (lbm_handle* h : b->cases) h->inited = false;
    b->failed = true;
    return st;
}

// after an odd number of batch steps every case's current buffer flips
static void batch_flip(lbm_batch* b, long long steps) {
    if (steps & 1)
        for (int c = 0; c < b->ncases; ++c) b->cases[c]->cur ^= 1;
}

// Time every tile shape of each class on the live state (all shapes give the
// same bits) and keep the fastest; the classes are timed one after the other.
static lbm_status batch_tune(lbm_batch* b, long long& done) {
    lbm_status st;
    const long long start = done;
    for (int cls = 0; cls < BATCH_NCLASS; ++cls) {
        if (!b->ncls[cls]) continue;
        long long s = start;
        double best = 1e300;
        for (int k = 0; k < BATCH_NCAND; ++k) {
            for (int w = 0; w < BATCH_TUNE_WARM; ++w, ++s)
                if ((st = batch_launch(b, cls, k, (int)(s & 1))) != LBM_OK) return st;
            double us = 1e300;
            for (int win = 0; win < BATCH_TUNE_WINDOWS; ++win) {
                LBM_BCUDA(b, cudaEventRecord(b->t0, b->bs[cls]));
                for (int w = 0; w < BATCH_TUNE_WINDOW; ++w, ++s)
                    if ((st = batch_launch(b, cls, k, (int)(s & 1))) != LBM_OK) return st;
                LBM_BCUDA(b, cudaEventRecord(b->t1, b->bs[cls]));
                LBM_BCUDA(b, cudaEventSynchronize(b->t1));
                float ms = 0.f;
                LBM_BCUDA(b, cudaEventElapsedTime(&ms, b->t0, b->t1));
                if (1e3 * ms / BATCH_TUNE_WINDOW < us) us = 1e3 * ms / BATCH_TUNE_WINDOW;
            }
            b->tuned_us[cls][k] = us;
            if (b->tuned_us[cls][k] < best) {
                best = b->tuned_us[cls][k];
                b->cand[cls] = k;
            }
        }
        done = s;
    }
    b->tuned = true;
    return LBM_OK;
}

// Capture BATCH_GRAPH_STEPS steps (parities 0, 1, ...) of both classes, each
// class a chain of launches on its own stream, the two chains independent.
static lbm_status batch_capture(lbm_batch* b) {
    cudaGraph_t g;
    LBM_BCUDA(b, cudaStreamBeginCapture(b->bs[0], cudaStreamCaptureModeThreadLocal));
    lbm_status st = batch_fork(b);
    if (st == LBM_OK) st = batch_run(b, 0, BATCH_GRAPH_STEPS);
    if (st == LBM_OK) st = batch_join(b);
    cudaError_t ce = cudaStreamEndCapture(b->bs[0], &g);
    if (st != LBM_OK) {
        if (ce == cudaSuccess) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        b->graph = nullptr;
        return bfail(b, LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    }
    return LBM_OK;
}

extern "C" {

lbm_status lbm_batch_create(int ncases, lbm_handle* const* cases, lbm_batch** out) {
    if (!out) return LBM_ERR_INVALID;
    *out = nullptr;
    if (ncases < 1 || ncases > BATCH_MAX_CASES || !cases) {
        fprintf(stderr, "lbm_batch_create: need 1 <= ncases <= %d and a case array\n",
                BATCH_MAX_CASES);
        return LBM_ERR_INVALID;
    }
    for (int c = 0; c < ncases; ++c) {
        const lbm_handle* h = cases[c];
        if (!h || !h->inited || h->device != cases[0]->device || h->stream != cases[0]->stream ||
            h->prm.storage != cases[0]->prm.storage) {
            fprintf(stderr, "lbm_batch_create: case %d is NULL, not initialised, or differs in "
                            "device, stream or storage from case 0\n", c);
            return LBM_ERR_INVALID;
        }
        for (int d = 0; d < c; ++d)
            if (cases[d] == h) {
                fprintf(stderr, "lbm_batch_create: case %d repeats case %d\n", c, d);
                return LBM_ERR_INVALID;
            }
    }
    // the graph replays fixed launches, so it has no per-step seed to give
    // the dithers of stochastic rounding
    if (cases[0]->prm.storage == LBM_STORE_BF16_SHIFTED_SR) {
        fprintf(stderr, "lbm_batch_create: LBM_STORE_BF16_SHIFTED_SR is not available in batches "
                        "(step such cases one by one)\n");
        return LBM_ERR_INVALID;
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->ncases = ncases;
    b->cases.assign(cases, cases + ncases);
    b->cls_of.resize(ncases);
    b->slot_of.resize(ncases);
    for (int c = 0; c < ncases; ++c) {
        const int cls = cases[c]->model.walls ? 1 : 0;
        b->cls_of[c] = cls;
        b->slot_of[c] = b->ncls[cls]++;
    }
    b->storage = cases[0]->prm.storage;
    b->device = cases[0]->device;
    b->user = cases[0]->stream;
    auto bad = [&](lbm_status st) {
        fprintf(stderr, "lbm_batch_create: %s\n", b->err);
        batch_release(b);
        delete b;
        return st;
    };
    if (cudaSetDevice(b->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->bs[0], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->bs[1], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess) {
        bfail(b, LBM_ERR_CUDA, "stream/event creation failed");
        return bad(LBM_ERR_CUDA);
    }
    b->table = new (std::nothrow) BatchTable[BATCH_NCLASS * BATCH_NCAND];
    if (!b->table) {
        bfail(b, LBM_ERR_OOM, "table allocation failed");
        return bad(LBM_ERR_OOM);
    }
    for (int cls = 0; cls < BATCH_NCLASS; ++cls)
        for (int k = 0; k < BATCH_NCAND; ++k) {
            BatchTable& T = b->tab(cls, k);
            memset(&T, 0, sizeof T);
            // tile height in nodes (16-bit kernels take LBM_NPT16_BATCH nodes per thread)
            const int th = BATCH_TY[k] * (b->storage == LBM_STORE_FP32 ? 1 : LBM_NPT16_BATCH);
            T.ncases = b->ncls[cls];
            long long tiles = 0;
            for (int c = 0; c < ncases; ++c) {
                if (b->cls_of[c] != cls) continue;
                const lbm_handle* h = cases[c];
                const int j = b->slot_of[c];
                CaseDesc& d = T.c[j];
                d.f[0] = h->f[0];
                d.f[1] = h->f[1];
                d.g[0] = h->g[0];
                d.g[1] = h->g[1];
                d.phiu = h->phiu;
                d.flag = h->flag;
                d.nx = h->nx;
                d.ny = h->ny;
                d.cur = h->cur;
                d.map0 = -1;
                d.m = h->model;
                T.tiles_x[j] = (h->nx + BATCH_TX[k] - 1) / BATCH_TX[k];
                T.tile0[j] = (int)tiles;
                tiles += (long long)T.tiles_x[j] * ((h->ny + th - 1) / th);
            }
            if (tiles >= (1LL << 31) - 1) {
                bfail(b, LBM_ERR_INVALID, "batch too large for one launch");
                return bad(LBM_ERR_INVALID);
            }
            T.tile0[T.ncases] = (int)tiles;
            // the tile list: (case, tile row << 16 | tile column), case-major
            std::vector<int2> list((size_t)tiles);
            size_t n = 0;
            for (int j = 0; j < T.ncases; ++j) {
                const int tx = T.tiles_x[j], ty = (T.c[j].ny + th - 1) / th;
                if (tx > 0xffff || ty > 0x7fff) {
                    bfail(b, LBM_ERR_INVALID, "a case has more than 65535 x 32767 tiles");
                    return bad(LBM_ERR_INVALID);
                }
                for (int r = 0; r < ty; ++r)
                    for (int q = 0; q < tx; ++q) list[n++] = make_int2(j, (r << 16) | q);
            }
            int2*& d = b->d_tiles[cls * BATCH_NCAND + k];
            if (tiles > 0) {
                if (cudaMalloc(&d, tiles * sizeof(int2)) != cudaSuccess ||
                    cudaMemcpy(d, list.data(), tiles * sizeof(int2), cudaMemcpyHostToDevice) !=
                        cudaSuccess) {
                    bfail(b, LBM_ERR_OOM, "tile list allocation failed");
                    return bad(LBM_ERR_OOM);
                }
            }
        }
    for (int c = 0; c < ncases; ++c) {
        b->node_count += (long long)cases[c]->N;
        if (cases[c]->prm.check_every > 0) b->check = true;
    }
    {
        // prefetch when a step's traffic exceeds the L2 threshold of the
        // single-case step (the classes run concurrently: their sum counts)
        int sms = 0, l2 = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess &&
            cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device) == cudaSuccess) {
            const bool st16 = b->storage != LBM_STORE_FP32;
            bool maps16 = st16 && LBM_TMA_PREFETCH && tensor_map_encoder() != nullptr;
            for (int c = 0; c < ncases; ++c)
                maps16 = maps16 && cases[c]->nx % 8 == 0 && cases[c]->nx >= BATCH_PF_BOX_X &&
                         cases[c]->ny >= BATCH_PF_BOX_Y;
            const double bytes = (st16 ? 92.0 : 160.0) * (double)b->node_count;
            const int thr = !st16 ? LBM_PREFETCH_L2X10 : maps16 ? LBM_PREFETCH16_TMA_L2X10 : LBM_PREFETCH16_L2X10;
            if (bytes * 10.0 >= (double)thr * l2) b->pf_ahead = LBM_BATCH_PF_PER10SM * sms / 10;
            // 16-bit batches prefetch through tensor maps: 8 per case (4 per
            // buffer), in device memory, indexed from the case table
            if (b->pf_ahead > 0 && maps16) {
                std::vector<CUtensorMap> maps((size_t)ncases * 8);
                bool ok = true;
                for (int c = 0; c < ncases && ok; ++c)
                    ok = encode_maps16(cases[c], 0, &maps[8 * c], BATCH_PF_BOX_X, BATCH_PF_BOX_Y) &&
                         encode_maps16(cases[c], 1, &maps[8 * c + 4], BATCH_PF_BOX_X, BATCH_PF_BOX_Y);
                if (ok && cudaMalloc(&b->d_maps, maps.size() * sizeof(CUtensorMap)) == cudaSuccess &&
                    cudaMemcpy(b->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                               cudaMemcpyHostToDevice) == cudaSuccess) {
                    for (int cls = 0; cls < BATCH_NCLASS; ++cls)
                        for (int k = 0; k < BATCH_NCAND; ++k) b->tab(cls, k).maps = b->d_maps;
                    for (int c = 0; c < ncases; ++c)
                        for (int k = 0; k < BATCH_NCAND; ++k)
                            b->tab(b->cls_of[c], k).c[b->slot_of[c]].map0 = 8 * c;
                } else {
                    if (b->d_maps) cudaFree(b->d_maps);
                    b->d_maps = nullptr;
                    // the per-thread requests' own threshold
                    if (bytes * 10.0 < (double)LBM_PREFETCH16_L2X10 * l2) b->pf_ahead = 0;
                }
            }
        }
    }
    // batch index of each class slot, for gathering the cases' flags
    for (int cls = 0; cls < BATCH_NCLASS; ++cls) {
        if (!b->ncls[cls]) continue;
        std::vector<int> idx;
        for (int c = 0; c < ncases; ++c)
            if (b->cls_of[c] == cls) idx.push_back(c);
        if (cudaMalloc(&b->d_slot[cls], idx.size() * sizeof(int)) != cudaSuccess ||
            cudaMemcpy(b->d_slot[cls], idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            bfail(b, LBM_ERR_OOM, "slot table allocation failed");
            return bad(LBM_ERR_OOM);
        }
    }
    if (cudaMalloc(&b->d_flags, ncases * sizeof(unsigned int)) != cudaSuccess) {
        bfail(b, LBM_ERR_OOM, "flag array allocation failed");
        return bad(LBM_ERR_OOM);
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    for (int k = 0; k < BATCH_NCLASS; ++k) cudaStreamSynchronize(b->bs[k]);
    batch_release(b);
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : "null batch"; }

lbm_status lbm_batch_info(const lbm_batch* b, int cls, int* ncases, int* tile_tx, int* tile_ty,
                          double* us_per_step, int* tuned) {
    if (!b || cls < 0 || cls >= BATCH_NCLASS) return LBM_ERR_INVALID;
    if (ncases) *ncases = b->ncls[cls];
    if (tile_tx) *tile_tx = BATCH_TX[b->cand[cls]];
    if (tile_ty)
        *tile_ty = BATCH_TY[b->cand[cls]] * (b->storage == LBM_STORE_FP32 ? 1 : LBM_NPT16_BATCH);
    if (us_per_step) *us_per_step = b->tuned_us[cls][b->cand[cls]];
    if (tuned) *tuned = b->tuned ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps) {
    if (!b) return LBM_ERR_INVALID;
    if (b->failed)
        return bfail(b, LBM_ERR_STATE, "lbm_batch_step: an earlier step call failed; re-initialise "
                                       "the cases and build a new batch");
    if (nsteps < 0) return bfail(b, LBM_ERR_INVALID, "lbm_batch_step: nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    for (int c = 0; c < b->ncases; ++c)
        if (!b->cases[c]->inited)
            return bfail(b, LBM_ERR_STATE, "lbm_batch_step: case %d is not initialised", c);
    LBM_BCUDA(b, cudaSetDevice(b->device));
    // order after earlier work on the cases' stream
    LBM_BCUDA(b, cudaEventRecord(b->ev_in, b->user));
    LBM_BCUDA(b, cudaStreamWaitEvent(b->bs[0], b->ev_in, 0));
    batch_sync_table(b);
    lbm_status st;
    if ((st = batch_fork(b)) != LBM_OK) return batch_abort(b, st);

    long long done = 0;
    // tune on the first call long enough: it runs tune_steps real steps
    const int tune_steps = BATCH_NCAND * BATCH_TUNE_PER_SHAPE;
    if (!b->tuned && nsteps >= tune_steps)
        if ((st = batch_tune(b, done)) != LBM_OK) return batch_abort(b, st);
    // an odd count so far: one more step so the graph starts at parity 0
    if ((done & 1) && done < nsteps) {
        if ((st = batch_run(b, done, done + 1)) != LBM_OK) return batch_abort(b, st);
        ++done;
    }
    if ((st = batch_join(b)) != LBM_OK) return batch_abort(b, st);
    // whole graph replays (BATCH_GRAPH_STEPS steps each, parity returns to 0)
    const long long reps = (nsteps - done) / BATCH_GRAPH_STEPS;
    if (reps > 0) {
        if (!b->graph && (st = batch_capture(b)) != LBM_OK) return batch_abort(b, st);
        for (long long r = 0; r < reps; ++r) {
            const cudaError_t ce = cudaGraphLaunch(b->graph, b->bs[0]);
            if (ce != cudaSuccess)
                return batch_abort(b, bfail(b, LBM_ERR_CUDA, "cudaGraphLaunch: %s",
                                            cudaGetErrorString(ce)));
        }
    }
    // the remainder, with parities continuing from 0 after the replays
    if (done + reps * BATCH_GRAPH_STEPS < nsteps) {
        if ((st = batch_fork(b)) != LBM_OK) return batch_abort(b, st);
        if ((st = batch_run(b, done + reps * BATCH_GRAPH_STEPS, nsteps)) != LBM_OK)
            return batch_abort(b, st);
        if ((st = batch_join(b)) != LBM_OK) return batch_abort(b, st);
    }
    // cases' current buffers (and with them the tables) follow
    batch_flip(b, nsteps);
    batch_sync_table(b);
    if (b->check) {
        // the cases' non-finite flags (set by any step of this call), gathered
        // and cleared on the device, then read on the host
        for (int cls = 0; cls < BATCH_NCLASS; ++cls)
            if (b->ncls[cls]) {
                const BatchTable& T = b->tab(cls, 0);
                k_batch_flags<<<(T.ncases + 127) / 128, 128, 0, b->bs[0]>>>(T, b->d_slot[cls],
                                                                            b->d_flags);
                LBM_BCUDA(b, cudaGetLastError());
            }
        std::vector<unsigned int> fl(b->ncases);
        LBM_BCUDA(b, cudaMemcpyAsync(fl.data(), b->d_flags, b->ncases * sizeof(unsigned int),
                                     cudaMemcpyDeviceToHost, b->bs[0]));
        LBM_BCUDA(b, cudaStreamSynchronize(b->bs[0]));
        for (int c = 0; c < b->ncases; ++c)
            if (fl[c] & 4u) {
                LBM_BCUDA(b, cudaEventRecord(b->ev_out, b->bs[0]));
                LBM_BCUDA(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
                return bfail(b, LBM_ERR_CUDA, "case %d: an index check of the debug build failed", c);
            }
        for (int c = 0; c < b->ncases; ++c)
            if (fl[c] && b->cases[c]->prm.check_every > 0) {
                LBM_BCUDA(b, cudaEventRecord(b->ev_out, b->bs[0]));
                LBM_BCUDA(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
                return bfail(b, LBM_ERR_NONFINITE,
                             "case %d produced a non-finite phi, u or p in this batch step", c);
            }
    }
    LBM_BCUDA(b, cudaEventRecord(b->ev_out, b->bs[0]));
    LBM_BCUDA(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Impact-case tooling: the spreading radius of Sec. III D (Fig. 8) and point
// probes of the fields, both evaluated on the device from the current state
// with the step's own arithmetic (phi by the same pull and sum, the fields by
// the same stencil and recovery), so they equal lbm_get_fields bit for bit at
// the nodes they touch.
// ---------------------------------------------------------------------------
namespace {

// One block scans row y: the last column left of xc and the first column
// right of xc where phi < 1/2 bound the liquid run through xc.
// out = [r, r_interp, x_left, x_right].
template <int ST>
__global__ void k_spreading_radius(const void* __restrict__ fs, int nx, int ny, int walls, int y,
                                   int xc, double* __restrict__ out) {
    __shared__ int s_left, s_right;
    const int N = nx * ny;
    if (threadIdx.x == 0) {
        s_left = -1;
        s_right = nx;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        if (x == xc) continue;
        const float phi = phi_at_st<ST, -1>(fs, N, x, y, nx, ny, walls);
        if (!(phi >= 0.5f)) {
            if (x < xc) atomicMax(&s_left, x);
            else atomicMin(&s_right, x);
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    auto phi_of = [&](int x) { return (double)phi_at_st<ST, -1>(fs, N, x, y, nx, ny, walls); };
    if (!(phi_of(xc) >= 0.5)) {
        out[0] = out[1] = 0.0;
        out[2] = out[3] = -1.0;
        return;
    }
    const int xl = s_left + 1, xr = s_right - 1;
    out[0] = 0.5 * (xr - xl + 1);
    // phi = 1/2 crossings by linear interpolation between the run's end nodes
    // and their gas neighbours; a run that reaches the grid edge ends half a
    // node beyond it
    double L = xl - 0.5, R = xr + 0.5;
    if (s_left >= 0) {
        const double a = phi_of(s_left), b = phi_of(xl);
        L = s_left + (0.5 - a) / (b - a);
    }
    if (s_right < nx) {
        const double a = phi_of(xr), b = phi_of(s_right);
        R = xr + (a - 0.5) / (a - b);
    }
    out[1] = 0.5 * (R - L);
    out[2] = xl;
    out[3] = xr;
}

// Fields at npts nodes (xy = x0, y0, x1, y1, ...), planes out[k * npts + j]
// for phi, rho, ux, uy, p.
template <int ST>
__global__ void k_probe(const void* __restrict__ fs, const void* __restrict__ gs, int nx, int ny,
                        Model m, const int* __restrict__ xy, int npts, double* __restrict__ out) {
    const int N = nx * ny;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < npts; j += gridDim.x * blockDim.x) {
        const int x = xy[2 * j], y = xy[2 * j + 1];
        float ph[3][3];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx)
                ph[dy + 1][dx + 1] = phi_at_st<ST, -1>(fs, N, fold_x(x + dx, nx),
                                                       fold_y(y + dy, ny, m.walls), nx, ny, m.walls);
        float f[9], g[9];
        pull18<ST>(fs, gs, N, make_nbr(x, y, nx, ny, m.walls), f, g);
        const float phi = ph[1][1];
        const Stencil st = stencil(phi, ph[1][2], ph[1][0], ph[2][1], ph[0][1], ph[2][2], ph[2][0],
                                   ph[0][0], ph[0][2]);
        const Macro M = macro_from(m, Pop<ST>::gmom(g), phi, st.gx, st.gy, st.lap);
        out[j] = phi;
        out[npts + j] = M.rho;
        out[2 * npts + j] = M.ux;
        out[3 * npts + j] = M.uy;
        out[4 * npts + j] = M.p;
    }
}

// Pressure averages inside r < r_in and outside r > r_out of (xc, yc) over
// the fields buffer (p is plane 4), with the minimum-image distance along
// periodic directions: block partials (sum in, count in, sum out, count out)
// into part, then one block folds them in a fixed order into res.
__global__ void __launch_bounds__(RED_THREADS)
    k_jump_partial(const double* __restrict__ fields, int nx, int ny, int periodic_y, double xc,
                   double yc, double r_in2, double r_out2, double* __restrict__ part) {
    __shared__ double s[4][RED_THREADS];
    const size_t N = (size_t)nx * ny;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t n = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; n < N;
         n += (size_t)gridDim.x * RED_THREADS) {
        double dx = (double)(n % nx) - xc, dy = (double)(n / nx) - yc;
        dx -= nx * rint(dx / nx);
        if (periodic_y) dy -= ny * rint(dy / ny);
        const double r2 = dx * dx + dy * dy, p = fields[4 * N + n];
        if (r2 < r_in2) {
            a[0] += p;
            a[1] += 1.0;
        } else if (r2 > r_out2) {
            a[2] += p;
            a[3] += 1.0;
        }
    }
    const int t = threadIdx.x;
    for (int k = 0; k < 4; ++k) s[k][t] = a[k];
    __syncthreads();
    for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
        if (t < h)
            for (int k = 0; k < 4; ++k) s[k][t] += s[k][t + h];
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = s[k][0];
}

__global__ void __launch_bounds__(RED_THREADS)
    k_jump_final(const double* __restrict__ part, int nb, double* __restrict__ res) {
    __shared__ double s[4][RED_THREADS];
    const int t = threadIdx.x;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = t; b < nb; b += RED_THREADS)
        for (int k = 0; k < 4; ++k) a[k] += part[4 * b + k];
    for (int k = 0; k < 4; ++k) s[k][t] = a[k];
    __syncthreads();
    for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
        if (t < h)
            for (int k = 0; k < 4; ++k) s[k][t] += s[k][t + h];
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < 4; ++k) res[k] = s[k][0];
}

}  // namespace

extern "C" {

lbm_status lbm_laplace_jump(lbm_handle* h, double xc, double yc, double r_in, double r_out,
                            double* dp) {
    if (!h) return LBM_ERR_INVALID;
    if (!dp) return fail(h, LBM_ERR_INVALID, "lbm_laplace_jump: NULL output");
    if (!h->inited) return fail(h, LBM_ERR_STATE, "lbm_laplace_jump before lbm_init");
    if (!(r_in > 0) || !(r_out >= r_in) || !std::isfinite(xc) || !std::isfinite(yc) ||
        !std::isfinite(r_out))
        return fail(h, LBM_ERR_INVALID, "lbm_laplace_jump: need finite centre and 0 < r_in <= r_out");
    LBM_CUDA(h, cudaSetDevice(h->device));
    double* buf = (double*)h->staging;
    lbm_status st = launch_step(h, true, buf);
    if (st != LBM_OK) return st;
    k_jump_partial<<<RED_BLOCKS, RED_THREADS, 0, h->stream>>>(buf, h->nx, h->ny, h->model.walls == 0,
                                                               xc, yc, r_in * r_in, r_out * r_out,
                                                               h->red_part);
    LBM_CUDA(h, cudaGetLastError());
    k_jump_final<<<1, RED_THREADS, 0, h->stream>>>(h->red_part, RED_BLOCKS, h->red_res);
    LBM_CUDA(h, cudaGetLastError());
    double r[4];
    LBM_CUDA(h, cudaMemcpyAsync(r, h->red_res, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (r[1] == 0.0 || r[3] == 0.0)
        return fail(h, LBM_ERR_INVALID, "lbm_laplace_jump: no node inside r_in or outside r_out");
    *dp = r[0] / r[1] - r[2] / r[3];
    return LBM_OK;
}

lbm_status lbm_spreading_radius(lbm_handle* h, int y, int xc, double* r, double* r_interp) {
    if (!h) return LBM_ERR_INVALID;
    if (!h->inited) return fail(h, LBM_ERR_STATE, "lbm_spreading_radius before lbm_init");
    if (y < 0 || y >= h->ny || xc < 0 || xc >= h->nx)
        return fail(h, LBM_ERR_INVALID, "lbm_spreading_radius: (xc, y) = (%d, %d) outside the grid",
                    xc, y);
    LBM_CUDA(h, cudaSetDevice(h->device));
    auto k = h->prm.storage == LBM_STORE_FP16_SHIFTED ? k_spreading_radius<ST_FP16>
             : is_bf16(h->prm.storage)                ? k_spreading_radius<ST_BF16>
                                                       : k_spreading_radius<ST_FP32>;
    k<<<1, 1024, 0, h->stream>>>(h->f[h->cur], h->nx, h->ny, h->model.walls, y, xc, h->red_res);
    LBM_CUDA(h, cudaGetLastError());
    double res[4];
    LBM_CUDA(h, cudaMemcpyAsync(res, h->red_res, sizeof res, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (r) *r = res[0];
    if (r_interp) *r_interp = res[1];
    return LBM_OK;
}

lbm_status lbm_probe(lbm_handle* h, int npts, const int* x, const int* y, double* phi, double* rho,
                     double* ux, double* uy, double* p) {
    if (!h) return LBM_ERR_INVALID;
    if (!h->inited) return fail(h, LBM_ERR_STATE, "lbm_probe before lbm_init");
    if (npts < 0 || (size_t)npts > h->N)
        return fail(h, LBM_ERR_INVALID, "lbm_probe: need 0 <= npts <= nx*ny, got %d", npts);
    if (npts == 0) return LBM_OK;
    if (!x || !y) return fail(h, LBM_ERR_INVALID, "lbm_probe: NULL coordinates");
    std::vector<int> xy(2 * (size_t)npts);
    for (int j = 0; j < npts; ++j) {
        if (x[j] < 0 || x[j] >= h->nx || y[j] < 0 || y[j] >= h->ny)
            return fail(h, LBM_ERR_INVALID, "lbm_probe: point %d = (%d, %d) outside the grid", j,
                        x[j], y[j]);
        xy[2 * j] = x[j];
        xy[2 * j + 1] = y[j];
    }
    LBM_CUDA(h, cudaSetDevice(h->device));
    // staging holds 80 B per node: 8 B of coordinates and 40 B of fields per point
    int* d_xy = (int*)h->staging;
    double* d_out = (double*)h->staging + h->N;
    LBM_CUDA(h, cudaMemcpyAsync(d_xy, xy.data(), xy.size() * sizeof(int), cudaMemcpyHostToDevice,
                                h->stream));
    auto k = h->prm.storage == LBM_STORE_FP16_SHIFTED ? k_probe<ST_FP16>
             : is_bf16(h->prm.storage)                ? k_probe<ST_BF16>
                                                       : k_probe<ST_FP32>;
    const int blocks = (npts + 127) / 128 < 1184 ? (npts + 127) / 128 : 1184;
    k<<<blocks, 128, 0, h->stream>>>(h->f[h->cur], h->g[h->cur], h->nx, h->ny, h->model, d_xy,
                                      npts, d_out);
    LBM_CUDA(h, cudaGetLastError());
    double* outs[5] = {phi, rho, ux, uy, p};
    for (int k5 = 0; k5 < 5; ++k5)
        if (outs[k5])
            LBM_CUDA(h, cudaMemcpyAsync(outs[k5], d_out + (size_t)k5 * npts, npts * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // extern "C"
