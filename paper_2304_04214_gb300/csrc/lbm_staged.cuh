// lbm_staged.cuh -- the fused step with its loads staged through shared memory
// by the tensor memory accelerator (TMA).
//
// Same arithmetic as step2_kernel (two x-adjacent cells per thread, packed
// FP32x2 collision), different data movement: a persistent grid walks tiles of
// 128 x-cells by 2 rows of one z-plane.  A producer warp issues, per tile, 19
// cp.async.bulk.tensor boxes (one per direction q, each shifted by -c_y and
// -c_z, one 16-byte granule of padding on both x ends to cover -c_x) into a
// ring of shared-memory stages; "full" mbarriers tell the four consumer warps
// that a stage has landed, "empty" mbarriers tell the producer that all four
// have read it.  DRAM latency is hidden by the copies in flight, not by
// resident warps, and no block-wide barrier sits in the tile loop.
// Interior rows 1 .. ny-2 only; the wall rows run in wall_kernel beside it.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbmk {

constexpr int SG_TX = 128;                 // cells along x per tile
constexpr int SG_TY = BY;                  // rows per tile (the wall path pairs rows too)
constexpr int SG_CONSUMERS = SG_TX / 2 * SG_TY;      // 4 warps, two cells per thread
constexpr int SG_THREADS = SG_CONSUMERS + 32;           // + the producer warp

template <class S>
struct Staged {
    using T = typename S::T;
    static constexpr int A = 16 / (int)sizeof(T);                     // x padding: one TMA granule
    static constexpr int BW = SG_TX + 2 * A;                          // box width (elements)
    static constexpr int BOX_BYTES = BW * SG_TY * (int)sizeof(T);     // bytes one box writes
    static constexpr int SLOT = (BOX_BYTES + 127) / 128 * 128;        // smem bytes per direction
    static constexpr int STAGE = 19 * SLOT;                           // smem bytes per tile
};
// dynamic shared memory of one block: the ring plus alignment slack
template <class S, int STAGES> constexpr int staged_smem_bytes() { return STAGES * Staged<S>::STAGE + 128; }

#ifndef LBM_SG_STAGES32
#define LBM_SG_STAGES32 3
#endif
#ifndef LBM_SG_STAGES16
#define LBM_SG_STAGES16 5
#endif
#ifndef LBM_SG_MINB32
#define LBM_SG_MINB32 3
#endif
#ifndef LBM_SG_MINB16
#define LBM_SG_MINB16 3
#endif
// Pipeline depth and resident blocks per SM per storage.
template <class S> struct StagedCfg {
    static constexpr int STAGES = LBM_SG_STAGES16, MINB = LBM_SG_MINB16;
};
template <> struct StagedCfg<StoreF32> {
    static constexpr int STAGES = LBM_SG_STAGES32, MINB = LBM_SG_MINB32;
};

template <class S>
struct StagedArgs {
    CUtensorMap tmap;        // 4-d map of the input lattice: (x, y, z, q), box (BW, SG_TY, 1, 1)
    StepArgs<S> s;
    int nxt, nyt, ntiles;    // interior tiles: x tiles, row pairs from row 1, z planes
};

// ---- PTX wrappers: mbarrier and the tensor copy ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `polls` polls (~2^22 by default; each poll may
// itself suspend for a while), so a copy that never lands ends in an error
// flag, not a hang.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int polls = 1 << 22) {
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Exercises that path: one block waits, with the same bounded wait, on a
// barrier that no copy and no thread completes, and raises the timeout flag
// the way the staged kernel does (read back by lbm_sync as LBM_ETIMEOUT).
__global__ void wait_timeout_probe_kernel(unsigned *flags, int polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(smem_u32(&bar), 0u, polls);
    if (!ok && threadIdx.x == 0) atomicOr(flags + 2, 1u);
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}

// Shared-memory loads of one or two stored populations, as FP32.
template <class S> __device__ __forceinline__ float lds1(const typename S::T *p) { return S::ld(p); }
template <class S> __device__ __forceinline__ float2 lds2(const typename S::T *p) { return S::ld2(p); }

template <class S, bool STATS>
__global__ void __launch_bounds__(SG_THREADS, StagedCfg<S>::MINB)
    staged_kernel(const __grid_constant__ StagedArgs<S> g) {
    using T = typename S::T;
    using G = Staged<S>;
    constexpr int STAGES = StagedCfg<S>::STAGES;
    extern __shared__ __align__(128) unsigned char sg_smem[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    const StepArgs<S> &a = g.s;
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nb = gridDim.x, b = blockIdx.x;
    const int my_tiles = b < g.ntiles ? (g.ntiles - 1 - b) / nb + 1 : 0;
    // stage ring at a 128-byte boundary (the launch adds 128 bytes of slack)
    const uint32_t sraw = smem_u32(sg_smem);
    const uint32_t smem0 = (sraw + 127u) & ~127u;
    unsigned char *const ring = sg_smem + (smem0 - sraw);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), SG_CONSUMERS / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    // the n-th tile of this block; every other step walks the tiles backwards
    auto tile_of = [&](int n) {
        const int t = b + n * nb;
        return a.reverse ? g.ntiles - 1 - t : t;
    };

    if (tid >= SG_CONSUMERS) {
        // ---- producer warp: one lane fills the ring ----
        if (tid == SG_CONSUMERS) {
            int n = 0;
            for (; n < my_tiles; ++n) {
                const int s = n % STAGES;
                if (n >= STAGES && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(n / STAGES - 1) & 1u)) {
                    atomicOr(a.flags + 2, 1u);
                    break;
                }
                const int t = tile_of(n);
                const int xt = t % g.nxt, r = t / g.nxt;
                const int yt = r % g.nyt, k = r / g.nyt;
                const int x = xt * SG_TX - G::A, y = 1 + yt * SG_TY;
                const uint32_t bar = smem_u32(&full[s]);
                mbar_expect_tx(bar, 19u * G::BOX_BYTES);
                const uint32_t dst = smem0 + s * G::STAGE;
#pragma unroll
                for (int q = 0; q < 19; ++q) {
                    int kz = k - CZ(q);
                    kz = kz < 0 ? kz + nz : (kz >= nz ? kz - nz : kz);
                    tma_load_4d(dst + q * G::SLOT, &g.tmap, x, y - CY(q), kz, q, bar);
                }
            }
            // copies still in flight land before the block may retire; a
            // drain wait that gives up raises the timeout flag (the step's
            // output is then invalid and lbm_sync reports LBM_ETIMEOUT)
            for (int m = n - STAGES > 0 ? n - STAGES : 0; m < n; ++m)
                if (!mbar_wait(smem_u32(&full[m % STAGES]), (uint32_t)(m / STAGES) & 1u))
                    atomicOr(a.flags + 2, 1u);
        }
        return;
    }

    // ---- consumer warps: (64, 2) threads, two cells each ----
    const int tx = tid % (SG_TX / 2), ty = tid / (SG_TX / 2);
    const int lane = tid & 31;
    const int plane = nx * ny;

    // interior tiles
    for (int n = 0; n < my_tiles; ++n) {
        const int s = n % STAGES;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&full[s]), (uint32_t)(n / STAGES) & 1u));
        if (!ok) {                                    // warp-uniform
            if (lane == 0) atomicOr(a.flags + 2, 1u);
            return;
        }
        const int t = tile_of(n);
        const int xt = t % g.nxt, r = t / g.nxt;
        const int yt = r % g.nyt, k = r / g.nyt;
        const int i0 = xt * SG_TX + 2 * tx;
        const int j = 1 + yt * SG_TY + ty;
        const T *st = reinterpret_cast<const T *>(ring + s * G::STAGE) + ty * G::BW + 2 * tx + G::A;
        V2 f[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const T *p = st + q * (G::SLOT / (int)sizeof(T));
            if (CX(q) == 0) f[q] = lds2<S>(p);
            else if (CX(q) > 0) f[q] = make_float2(lds1<S>(p - 1), lds1<S>(p));
            else f[q] = make_float2(lds1<S>(p + 1), lds1<S>(p + 2));
        }
        // sources outside the box: periodic x wraps, the outlet copies its own column
        if (i0 + 2 == nx && a.inlet) {
#pragma unroll
            for (int q = 0; q < 19; ++q)
                if (CX(q) < 0) f[q].y = lds1<S>(st + q * (G::SLOT / (int)sizeof(T)) + 1);
        }
        // this warp has read stage s.  The next tensor copy into it writes
        // through the async proxy: the proxy fence orders these generic-proxy
        // reads before it (the mbarrier release / acquire alone does not).
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty[s]));

        const bool valid = i0 < nx && j < ny - 1;
        if (!a.inlet && (i0 == 0 || i0 + 2 == nx)) {
#pragma unroll
            for (int q = 0; q < 19; ++q) {
                if (CX(q) == 0) continue;
                int kz = k - CZ(q);
                kz = kz < 0 ? kz + nz : (kz >= nz ? kz - nz : kz);
                const typename S::T *row = a.in[q] + (kz * ny + j - CY(q)) * nx;
                if (CX(q) > 0 && i0 == 0) f[q].x = S::ld(row + nx - 1);
                if (CX(q) < 0 && i0 + 2 == nx) f[q].y = S::ld(row);
            }
        }
        rowbase_decode<S>(a, f, j);
        if (a.inlet && i0 == 0 && valid) {             // the lo cell is an inlet cell
            float fl[19];
#pragma unroll
            for (int q = 0; q < 19; ++q) fl[q] = f[q].x;
            inlet_rebuild<S>(a, fl, j, k);
#pragma unroll
            for (int q = 0; q < 19; ++q) f[q].x = fl[q];
        }
        V2 ux, uy, uz;
        collide_mrt2<S::SHIFTED>(f, pair_tau0(a, i0), a.csm18, ux, uy, uz);
        if (!valid) continue;
        const int c = (k * ny + j) * nx + i0;
        rowbase_encode<S>(a, f, j);
#pragma unroll
        for (int q = 0; q < 19; ++q) S::st2(a.out[q] + c, f[q]);
        if (STATS) {
            const long long N = (long long)plane * nz;
            *reinterpret_cast<float2 *>(a.ubuf + c) = ux;
            *reinterpret_cast<float2 *>(a.ubuf + N + c) = uy;
            *reinterpret_cast<float2 *>(a.ubuf + 2 * N + c) = uz;
        }
        if (a.check) {
            const V2 uu = vfma(ux, ux, vfma(uy, uy, uz * uz));
            if (!(uu.x < 0.09f) || !(uu.y < 0.09f)) atomicAdd(a.flags + 1, 1u);   // also catches NaN
        }
    }
}

}  // namespace lbmk
