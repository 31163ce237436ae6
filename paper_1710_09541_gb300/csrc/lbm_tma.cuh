// lbm_tma.cuh -- the step kernel with TMA-staged tiles (sm_103a).
//
// Same arithmetic as k_step (lbm_kernels.cuh), different data movement: a
// persistent CTA per SM walks the grid's TX x TY tiles.  While it collides
// tile k, the bulk tensor engine (cp.async.bulk.tensor, completion tracked by
// an mbarrier) copies tile k+1 into the other shared-memory stage:
//   f box  [9][TY+4][TX+8]  rows y0-2 .. y0+TY+1, columns x0-4 .. x0+TX+3
//          (the pulls of the tile plus its one-node phi ring; x starts 16-byte
//          aligned, 4 columns early)
//   g box  [9][TY+2][TX+8]  rows y0-1 .. y0+TY (the pulls of the tile)
//   phi u  [2][TY][TX]      the previous step's (phi u) of the tile
// The copies fill coordinates outside the grid with zeros; tiles on a
// periodic edge patch those halo entries from global memory after the copy.
// Every mbarrier wait is bounded; a timeout sets bit 1 of the status flag and
// the block returns after one more bounded wait on each stage with a copy in
// flight (the late one included).  A handle whose step reported a timeout
// must be destroyed: its state is undefined.
#pragma once
#include <cuda.h>

#include "lbm_kernels.cuh"
#include "lbm_store.cuh"

namespace lbmpf {

constexpr long long TMA_WAIT_LIMIT = 1LL << 22;  // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit = TMA_WAIT_LIMIT) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Self-test of the bounded wait: an mbarrier armed for 16 transaction bytes
// that no copy will deliver (none is issued, so nothing is in flight), then
// the same bounded wait the staged kernel uses, with a short limit.  A wait
// that gives up sets bit 1 of *flag (as in the staged kernel) and the block
// returns.
__global__ void k_wait_selftest(unsigned int* flag, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_arrive_expect_tx(&bar, 16);
    if (!mbar_wait_bounded(&bar, 0, limit)) atomicOr(flag, 2u);
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int TX, int TY>
struct TmaTile {
    static constexpr int FW = TX + 8;  // box row length in floats
    static constexpr int FH = TY + 4;  // f box rows
    static constexpr int GH = TY + 2;  // g box rows
    static constexpr uint32_t F_BYTES = 9u * FH * FW * 4u;
    static constexpr uint32_t G_BYTES = 9u * GH * FW * 4u;
    static constexpr uint32_t U_BYTES = 2u * TY * TX * 4u;
    static constexpr uint32_t COPY_BYTES = F_BYTES + G_BYTES + U_BYTES;  // per stage
    static constexpr size_t pad(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t F_OFF = 0;
    static constexpr size_t G_OFF = pad(F_BYTES);
    static constexpr size_t U_OFF = G_OFF + pad(G_BYTES);
    static constexpr size_t STAGE = U_OFF + pad(U_BYTES);
    static constexpr int PW = TX + 2, PH = TY + 2;  // phi on tile + ring
    static constexpr size_t PHI_OFF = 2 * STAGE;
    static constexpr size_t BAR_OFF = pad(PHI_OFF + size_t(PW) * PH * 4);
    static constexpr size_t SMEM = BAR_OFF + 128 + 128;  // + alignment slack
    static_assert(FW % 4 == 0, "TMA rows must be a multiple of 16 bytes");
    static_assert(COPY_BYTES < (1u << 20), "mbarrier transaction count");
};

// Pull of one node from a shared-memory box laid out [9][rows][FW]; (c, r) is
// the node's own position in the box.  Same association order and wall rule as
// pull9 (lbm_kernels.cuh).
template <int FW, int ROWS>
__device__ __forceinline__ void pull9_smem(const float* B, int c, int r, bool lo, bool hi,
                                           float v[9]) {
    constexpr int P = ROWS * FW;
    const int o = r * FW + c;
    v[0] = B[o];
    v[1] = B[P + o - 1];
    v[3] = B[3 * P + o + 1];
    v[2] = lo ? B[4 * P + o] : B[2 * P + o - FW];
    v[4] = hi ? B[2 * P + o] : B[4 * P + o + FW];
    v[5] = lo ? B[7 * P + o] : B[5 * P + o - FW - 1];
    v[6] = lo ? B[8 * P + o] : B[6 * P + o - FW + 1];
    v[7] = hi ? B[5 * P + o] : B[7 * P + o + FW + 1];
    v[8] = hi ? B[6 * P + o] : B[8 * P + o + FW - 1];
}

template <int TX, int TY, int NT, int WALLS>
__global__ void __launch_bounds__(NT, 1)
    k_step_tma(const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_g,
               const __grid_constant__ CUtensorMap tm_u, const float* __restrict__ fs,
               const float* __restrict__ gs, float* __restrict__ fd, float* __restrict__ gd,
               float* __restrict__ phiu, unsigned int* __restrict__ flag, int nx, int ny,
               int tiles_x, int ntiles, Model m) {
    m.walls = WALLS;
    using T = TmaTile<TX, TY>;
    constexpr int FW = T::FW, FH = T::FH, GH = T::GH, PW = T::PW, PH = T::PH;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bulk tensor copies land on 128-byte aligned addresses (SMEM has 128 B slack)
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + T::BAR_OFF);
    float* sphi = reinterpret_cast<float*>(smem + T::PHI_OFF);
    const int tid = threadIdx.x;
    const size_t N = (size_t)nx * ny;
    const bool periodic_y = !m.walls;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](int t, int s) {
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        unsigned char* st = smem + s * T::STAGE;
        mbar_arrive_expect_tx(&bar[s], T::COPY_BYTES);
        tma_load_3d(st + T::F_OFF, &tm_f, &bar[s], x0 - 4, y0 - 2, 0);
        tma_load_3d(st + T::G_OFF, &tm_g, &bar[s], x0 - 4, y0 - 1, 0);
        tma_load_3d(st + T::U_OFF, &tm_u, &bar[s], x0, y0, 0);
    };

    const int stride = gridDim.x;
    int t = blockIdx.x;
    if (tid == 0) {
        if (t < ntiles) issue(t, 0);
        if (t + stride < ntiles) issue(t + stride, 1);
    }
    for (int k = 0; t < ntiles; ++k, t += stride) {
        const int s = k & 1;
        const bool got = mbar_wait_bounded(&bar[s], (k >> 1) & 1);
        if (__syncthreads_or(!got)) {
            // a copy never completed: report, wait (bounded) once more for
            // the late stage's own copy and for the other stage's copy if one
            // is in flight, and leave
            if (tid == 0) {
                atomicOr(flag, 2u);
                mbar_wait_bounded(&bar[s], (k >> 1) & 1);
                if (t + stride < ntiles) mbar_wait_bounded(&bar[s ^ 1], ((k + 1) >> 1) & 1);
            }
            return;
        }
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        unsigned char* st = smem + s * T::STAGE;
        float* F = reinterpret_cast<float*>(st + T::F_OFF);
        float* G = reinterpret_cast<float*>(st + T::G_OFF);
        const float* U = reinterpret_cast<const float*>(st + T::U_OFF);

        // periodic edges: replace the zero fill outside the grid with the
        // wrapped values (walls: rows outside the grid are never read)
        const bool edge_x = (x0 - 2 < 0) || (x0 + TX + 2 > nx);
        const bool edge_y = periodic_y && ((y0 - 2 < 0) || (y0 + TY + 2 > ny));
        if (edge_x || edge_y) {
            constexpr int CW = TX + 4;  // box columns 2 .. TX+5 are read
            for (int e = tid; e < 9 * FH * CW; e += NT) {
                const int i = e / (FH * CW), rem = e % (FH * CW);
                const int r = rem / CW, c = 2 + rem % CW;
                const int gx = x0 - 4 + c, gy = y0 - 2 + r;
                const bool ox = gx < 0 || gx >= nx, oy = gy < 0 || gy >= ny;
                if ((ox || oy) && (periodic_y || !oy))
                    F[(i * FH + r) * FW + c] =
                        __ldg(fs + i * N + (size_t)fold_y(gy, ny, 0) * nx + fold_x(gx, nx));
            }
            constexpr int GC = TX + 2;  // g box columns 3 .. TX+4 are read
            for (int e = tid; e < 9 * GH * GC; e += NT) {
                const int i = e / (GH * GC), rem = e % (GH * GC);
                const int r = rem / GC, c = 3 + rem % GC;
                const int gx = x0 - 4 + c, gy = y0 - 1 + r;
                const bool ox = gx < 0 || gx >= nx, oy = gy < 0 || gy >= ny;
                if ((ox || oy) && (periodic_y || !oy))
                    G[(i * GH + r) * FW + c] =
                        __ldg(gs + i * N + (size_t)fold_y(gy, ny, 0) * nx + fold_x(gx, nx));
            }
            __syncthreads();
        }

        // phi (Eq. 12) on the tile and its ring; at a wall the ring row takes
        // the first/last row's value (mirror ghost)
        for (int pi = tid; pi < PW * PH; pi += NT) {
            const int px = pi % PW - 1, py = pi / PW - 1;
            int gy = y0 + py, ry = py;
            if (m.walls && (gy < 0 || gy >= ny)) {
                const int cy = gy < 0 ? 0 : ny - 1;
                ry += cy - gy;
                gy = cy;
            }
            float v[9];
            pull9_smem<FW, FH>(F, px + 4, ry + 2, m.walls && gy == 0, m.walls && gy == ny - 1, v);
            sphi[pi] = sum9(v);
        }
        __syncthreads();

        for (int q = tid; q < TX * TY; q += NT) {
            const int lx = q % TX, ly = q / TX;
            const int x = x0 + lx, y = y0 + ly;
            if (x >= nx || y >= ny) continue;
            const bool lo = m.walls && y == 0, hi = m.walls && y == ny - 1;
            float f[9], g[9];
            pull9_smem<FW, FH>(F, lx + 4, ly + 2, lo, hi, f);
            pull9_smem<FW, GH>(G, lx + 4, ly + 1, lo, hi, g);
            const float* sp = sphi + (ly + 1) * PW + (lx + 1);
            const float phi = sp[0];
            const Stencil stc = stencil(phi, sp[1], sp[-1], sp[PW], sp[-PW], sp[PW + 1], sp[PW - 1],
                                        sp[-PW - 1], sp[-PW + 1]);
            const Macro M = macroscopic(m, g, phi, stc.gx, stc.gy, stc.lap);
            if (!isfinite(add(add(phi, M.ux), add(M.uy, M.p)))) report_nonfinite(flag);
            const float2 prev = make_float2(U[ly * TX + lx], U[TX * TY + ly * TX + lx]);
            const float2 now = collide(m, f, g, phi, stc, M, prev);
            const size_t n = (size_t)y * nx + x;
            phiu[n] = now.x;
            phiu[N + n] = now.y;
            Pop<ST_FP32>::stfg(fd, gd, (int)N, (int)n, f, g, phi);
        }
        // the stage is read (and on edges written) through the generic proxy;
        // order that before the next bulk copy into it
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && t + 2 * stride < ntiles) issue(t + 2 * stride, s);
    }
}

// ---------------------------------------------------------------------------
// The step with 16-bit storage (Shifted16) and TMA-staged tiles: one TX x TY
// tile per CTA, many CTAs per SM.  Thread 0 copies the tile's pulls and its
// one-node phi ring into shared memory with two bulk tensor copies:
//   word box [8][TY+4][TX+8]  the (f_i, g_i) code words of the 8 moving
//             directions, rows y0-2 .. y0+TY+1, columns x0-4 .. x0+TX+3
//   f_0 box  [TY+2][TX+8]     rows y0-1 .. y0+TY, same columns
// (x starts 4 columns early so it is 16-byte aligned).  Every pull is then a
// shared-memory load at a fixed offset from the node's slot, so the pulls of
// the tile and of the ring need no address arithmetic and no wrap logic: the
// copies fill coordinates outside the grid with zeros, and tiles on a
// periodic edge patch those entries with the wrapped values from global
// memory before the pulls.  The arithmetic is the shared tile body's (same
// functions, same order), so the results equal the direct-load kernel's bit
// for bit.  The mbarrier wait is bounded; a timeout sets bit 1 of the status
// flag, the CTA waits (bounded) once more for its copies and returns.
// ---------------------------------------------------------------------------
template <int TX, int TY>
struct Tma16Tile {
    static constexpr int BW = TX + 8;   // box row length (words)
    static constexpr int WH = TY + 4;   // word box rows
    static constexpr int FH = TY + 2;   // f_0 box rows
    static constexpr int WP = WH * BW;  // one direction's plane in the word box
    static constexpr uint32_t W_BYTES = 8u * WP * 4u;
    static constexpr uint32_t F_BYTES = uint32_t(FH) * BW * 4u;
    static constexpr uint32_t COPY_BYTES = W_BYTES + F_BYTES;
    static_assert(BW % 4 == 0 && (W_BYTES % 128) == 0, "16-byte rows, 128-byte aligned f_0 box");
    static_assert(COPY_BYTES < (1u << 20), "mbarrier transaction count");
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// Pull of one node's 8 moving code words from the word box; o = the node's
// slot (row * BW + column).  lo / hi: the node sits on the wall at y = -1/2 /
// y = ny - 1/2 (half-way bounce-back: the link returns the node's own word of
// the opposite direction); top_open: the node is the top row under the open
// top (its c_y = -1 links pull from its own row).
template <int BW, int WP>
__device__ __forceinline__ void pull_words_smem(const unsigned int* B, int o, bool lo, bool hi,
                                                bool top_open, unsigned int w[9]) {
    // plane k - 1 holds direction k
    w[1] = B[0 * WP + o - 1];
    w[3] = B[2 * WP + o + 1];
    if (lo || hi || top_open) {
        const int up = top_open ? 0 : BW;  // row the c_y = -1 links pull from
        w[2] = lo ? B[3 * WP + o] : B[1 * WP + o - BW];
        w[4] = hi ? B[1 * WP + o] : B[3 * WP + o + up];
        w[5] = lo ? B[6 * WP + o] : B[4 * WP + o - BW - 1];
        w[6] = lo ? B[7 * WP + o] : B[5 * WP + o - BW + 1];
        w[7] = hi ? B[4 * WP + o] : B[6 * WP + o + up + 1];
        w[8] = hi ? B[5 * WP + o] : B[7 * WP + o + up - 1];
    } else {
        w[2] = B[1 * WP + o - BW];
        w[4] = B[3 * WP + o + BW];
        w[5] = B[4 * WP + o - BW - 1];
        w[6] = B[5 * WP + o - BW + 1];
        w[7] = B[6 * WP + o + BW + 1];
        w[8] = B[7 * WP + o + BW - 1];
    }
}

// WALLS: 0 periodic in y, 1 a wall at y = 0 and the kind of top read from
// m.walls (closed: 1, open: 2).  The same residency as the direct-load
// 16-bit kernels.
template <int TX, int TY, int ST, int WALLS>
__global__ void __launch_bounds__(TX* TY, (WALLS == 0 ? 9 : 10))
    k_step16_tma(const __grid_constant__ CUtensorMap tm_w, const __grid_constant__ CUtensorMap tm_f0,
                 const void* __restrict__ fs, const void* __restrict__ gs, void* __restrict__ fd,
                 void* __restrict__ gd, float* __restrict__ phiu, unsigned int* __restrict__ flag,
                 int nx, int ny, Model m) {
    using P = Pop<ST>;
    using T = Tma16Tile<TX, TY>;
    constexpr int BW = T::BW, WH = T::WH, WP = T::WP;
    __shared__ __align__(128) unsigned int sw[8 * WP];
    __shared__ __align__(128) float sf0[T::FH * BW];
    __shared__ float sphi[TY + 2][TX + 2];
    __shared__ __align__(8) uint64_t bar;
    if (WALLS == 0) m.walls = 0;
    const int walls = m.walls;
    const bool open_top = walls == 2;
    const int N = nx * ny;  // 20 N < 2^31 (checked at create)
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < nx) && (y < ny);

    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    griddep_wait();
    griddep_launch();
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, T::COPY_BYTES);
        tma_load_3d(sw, &tm_w, &bar, x0 - 4, y0 - 2, 0);
        tma_load_2d(sf0, &tm_f0, &bar, x0 - 4, y0 - 1);
    }
    // the node's own loads go out while the copies are in flight
    float2 prev = make_float2(0.f, 0.f);
    unsigned short g0 = 0;
    if (active) {
        prev = make_float2(phiu[y * nx + x], phiu[N + y * nx + x]);
        g0 = __ldg(static_cast<const unsigned short*>(gs) + (y * nx + x));
    }
    const bool got = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!got)) {
        if (tid == 0) {
            atomicOr(flag, 2u);
            mbar_wait_bounded(&bar, 0);  // the late copies may still land
        }
        return;
    }

    // periodic edges: the entries the pulls read outside the grid take the
    // wrapped values (walls: rows outside the grid are never read)
    const bool edge_x = (x0 - 2 < 0) || (x0 + TX + 2 > nx);
    const bool edge_y = walls == 0 && ((y0 - 2 < 0) || (y0 + TY + 2 > ny));
    if (edge_x || edge_y) {
        const unsigned int* W = P::pw(fs, N);
        constexpr int CW = TX + 4;  // box columns 2 .. TX+5 are read
        for (int e = tid; e < 8 * WH * CW; e += TX * TY) {
            const int k = e / (WH * CW), rem = e - k * (WH * CW);
            const int r = rem / CW, c = 2 + rem % CW;
            const int gx = x0 - 4 + c, gy = y0 - 2 + r;
            const bool ox = gx < 0 || gx >= nx, oy = gy < 0 || gy >= ny;
            if ((ox || oy) && (walls == 0 || !oy))
                sw[k * WP + r * BW + c] = __ldg(W + (k * N + fold_y(gy, ny, 0) * nx + fold_x(gx, nx)));
        }
        const float* F0 = static_cast<const float*>(fs);
        constexpr int CF = TX + 2;  // f_0 box columns 3 .. TX+4 are read
        for (int e = tid; e < T::FH * CF; e += TX * TY) {
            const int r = e / CF, c = 3 + e % CF;
            const int gx = x0 - 4 + c, gy = y0 - 1 + r;
            const bool ox = gx < 0 || gx >= nx, oy = gy < 0 || gy >= ny;
            if ((ox || oy) && (walls == 0 || !oy))
                sf0[r * BW + c] = __ldg(F0 + (fold_y(gy, ny, 0) * nx + fold_x(gx, nx)));
        }
        __syncthreads();
    }

    // phi (Eq. 12) of a tile or ring slot (lx, ly), -1 <= lx <= TX,
    // -1 <= ly <= TY: at a wall the ghost row is the edge row (mirror), and
    // a slot below or above the grid takes the edge row's phi
    auto phi_slot = [&](int lx, int ly, unsigned int w[9], float& f0) {
        int gy = y0 + ly;
        if (walls && (gy < 0 || gy >= ny)) gy = gy < 0 ? 0 : ny - 1;
        int br = gy - y0 + 2;  // word box row
#if LBM_DEBUG_CHECKS
        // the slot and its pulls stay inside the boxes: rows br - 1 .. br + 1
        // of the word box, columns lx + 3 .. lx + 5
        if (br < 1 || br > TY + 2 || lx < -1 || lx > TX) {
            atomicOr(flag, 4u);
            br = 2;
            lx = 0;
        }
#endif
        const bool lo = walls && gy == 0, hi = walls && !open_top && gy == ny - 1;
        const bool top = open_top && gy == ny - 1;
        pull_words_smem<BW, WP>(sw, br * BW + lx + 4, lo, hi, top, w);
        f0 = sf0[(br - 1) * BW + lx + 4];
        float h[9];
        h[0] = f0;
#pragma unroll
        for (int i = 1; i < 9; ++i) h[i] = P::C::to_f(P::lo(w[i]));
        return P::phi_of(h);
    };
    unsigned int w[9];
    float f0;
    sphi[ty + 1][tx + 1] = phi_slot(tx, ty, w, f0);
    for (int r = tid; r < Ring<TX, TY>::count; r += TX * TY) {
        int lx, ly;
        Ring<TX, TY>::pos(r, lx, ly);
        unsigned int wr[9];
        float f0r;
        sphi[ly + 1][lx + 1] = phi_slot(lx, ly, wr, f0r);
    }
    __syncthreads();
    if (!active) return;

    float h[9], k[9];
    h[0] = f0;
    k[0] = P::C::to_f(g0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        h[i] = P::C::to_f(P::lo(w[i]));
        k[i] = P::C::to_f(P::hi(w[i]));
    }
    const int lx = tx + 1, ly = ty + 1;
    const float phi = sphi[ly][lx];
    const Stencil st = stencil(phi, sphi[ly][lx + 1], sphi[ly][lx - 1], sphi[ly + 1][lx],
                               sphi[ly - 1][lx], sphi[ly + 1][lx + 1], sphi[ly + 1][lx - 1],
                               sphi[ly - 1][lx - 1], sphi[ly - 1][lx + 1]);
    const Macro M = macro_from(m, P::gmom(k), phi, st.gx, st.gy, st.lap);
    if (!isfinite(add(add(phi, M.ux), add(M.uy, M.p)))) report_nonfinite(flag);
    const float2 now = collide_code<P>(m, h, k, phi, st, M, prev);
    const int n = y * nx + x;
    phiu[n] = now.x;
    phiu[N + n] = now.y;
    P::stfg(fd, gd, N, n, h, k, phi);
}

}  // namespace lbmpf
