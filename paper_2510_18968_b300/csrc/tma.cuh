// tma.cuh -- tile loads by the tensor memory accelerator (TMA) for the FP32
// stencil kernels: a tensor map of a primitive-field array (x, y, z, field)
// or of one current component (x, y, z), one bulk tensor copy per tile into
// shared memory, completion on an mbarrier.  sm_100-family PTX
// (cp.async.bulk.tensor, mbarrier expect_tx / try_wait).
//
// Alignment contract (checked by make_tile_map and by the caller): the
// array base and every stride are multiples of 16 bytes (the grid's x pitch
// is rounded up to 4 cells), a box's x extent is a multiple of 4 floats, and
// the x coordinate of every copy is a multiple of 4.  A box may run past the
// end of the array: those elements are filled with zeros and never read.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace rmhd {

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of the barrier: false after `limit`
// polls (each poll may itself suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y,
                                            int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y,
                                            int z, int f, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(f),
        "r"(smem_u32(bar))
        : "memory");
}

// polls of a tile wait before the kernel gives up and reports (a tile
// arrives in microseconds; this bound is seconds)
constexpr unsigned TILE_WAIT_POLLS = 1u << 24;

// Host: a tiled tensor map of nf FP32 fields (nf = 0: one field, rank 3)
// of the padded grid (px, py, pz) starting at base, box {bx, by, bz(, nf)}.
// Returns false if the driver refuses it (alignment, sizes).
bool make_tile_map(CUtensorMap *map, const float *base, int px, int py, int pz,
                   long long field_stride, int nf, int bx, int by, int bz);

// host: count of flux-kernel launches that used tile copies (testing)
extern std::atomic<long long> g_tile_copy_launches;

} // namespace rmhd
