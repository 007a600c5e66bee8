// batch.cu -- many meshes evaluated and solved together.  A batch copies the
// resident state of already uploaded meshes into concatenated arrays: each
// mesh's source nodes start on a tile boundary, so a work item of the pair
// kernels (a block of one mesh's targets and that mesh's tile range) never
// mixes meshes.
#include <vector>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

__global__ void k_offset_tris(int32_t* __restrict__ tris, int64_t m, int32_t voff)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < 3 * m) tris[j] += voff;
}

}  // namespace

int batch_build(Ctx* ctx, Batch* b, lsm_mesh* const* meshes, int n, cudaStream_t st)
{
    b->ctx = ctx;
    b->nmesh = n;
    std::vector<int64_t> voff(n + 1, 0), toff(n + 1, 0), tileoff(n + 1, 0);
    for (int i = 0; i < n; i++) {
        const Mesh* me = &meshes[i]->m;
        if (me->ctx != ctx) {
            ctx->err = "batch: every mesh must belong to this context";
            return LSM_E_INVALID_ARG;
        }
        if (me->sigx) {
            ctx->err = "batch: meshes with a target-dependent sigma are solved one by one";
            return LSM_E_INVALID_ARG;
        }
        if (me->tris6) {
            ctx->err = "batch: meshes of quadratic patches are solved one by one";
            return LSM_E_INVALID_ARG;
        }
        voff[i + 1] = voff[i] + me->nv;
        toff[i + 1] = toff[i] + me->m;
        tileoff[i + 1] = tileoff[i] + me->ntiles;
    }
    if (voff[n] >= ((int64_t)1 << 31) || tileoff[n] * kTile >= ((int64_t)1 << 31)) {
        ctx->err = "batch: too many vertices or source nodes (limit 2^31)";
        return LSM_E_INVALID_ARG;
    }
    b->nv = voff[n];
    b->m = toff[n];
    b->ntiles = tileoff[n];
    b->tri_off = toff;
    const size_t nsrc = (size_t)b->ntiles * kTile;
    auto alloc = [&](auto** p, size_t count) -> bool {
        using T = std::remove_pointer_t<std::remove_reference_t<decltype(*p)>>;
        if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) return false;
        b->bytes += count * sizeof(T);
        return true;
    };
    if (!alloc(&b->verts, 3 * b->nv) || !alloc(&b->tris, 3 * b->m) || !alloc(&b->tri_sigma, b->m) ||
        !alloc(&b->vpn, 3 * b->nv) || !alloc(&b->tri_mesh, b->m) || !alloc(&b->s32_pos, nsrc) ||
        !alloc(&b->s32_nw, nsrc) || !alloc(&b->s32_lo, nsrc) || !alloc(&b->s32_nwlo, nsrc) ||
        !alloc(&b->s64_pos, nsrc) || !alloc(&b->s64_nw, nsrc) || !alloc(&b->tile_lo, b->ntiles) ||
        !alloc(&b->tile_hi, b->ntiles) || !alloc(&b->tile_chi, b->ntiles) || !alloc(&b->tile_clo, b->ntiles) ||
        !alloc(&b->mesh_tiles, n)) {
        cudaGetLastError();
        ctx->err = "batch: out of device memory";
        return LSM_E_OOM;
    }
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    std::vector<int32_t> tri_mesh((size_t)b->m);
    std::vector<int2> mt(n);
    for (int i = 0; i < n; i++) {
        const Mesh* me = &meshes[i]->m;
        const size_t so = (size_t)tileoff[i] * kTile;
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->verts + 3 * voff[i], me->verts, sizeof(double) * 3 * me->nv, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->vpn + 3 * voff[i], me->vpn, sizeof(double) * 3 * me->nv, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->tris + 3 * toff[i], me->tris, sizeof(int32_t) * 3 * me->m, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->tri_sigma + toff[i], me->tri_sigma, sizeof(double) * me->m, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->s32_pos + so, me->s32_pos, sizeof(float4) * me->ntiles * kTile, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->s32_nw + so, me->s32_nw, sizeof(float4) * me->ntiles * kTile, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->s32_lo + so, me->s32_lo, sizeof(float4) * me->ntiles * kTile, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->s32_nwlo + so, me->s32_nwlo, sizeof(float4) * me->ntiles * kTile, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->s64_pos + so, me->s64_pos, sizeof(double4_32a) * me->ntiles * kTile, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->s64_nw + so, me->s64_nw, sizeof(double4_32a) * me->ntiles * kTile, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->tile_lo + tileoff[i], me->tile_lo, sizeof(float4) * me->ntiles, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->tile_hi + tileoff[i], me->tile_hi, sizeof(float4) * me->ntiles, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->tile_chi + tileoff[i], me->tile_chi, sizeof(float4) * me->ntiles, dd, st));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->tile_clo + tileoff[i], me->tile_clo, sizeof(float4) * me->ntiles, dd, st));
        if (voff[i] > 0) {
            k_offset_tris<<<(unsigned)((3 * me->m + 255) / 256), 256, 0, st>>>(b->tris + 3 * toff[i], me->m,
                                                                             (int32_t)voff[i]);
            LSM_LAUNCHED(ctx);
        }
        for (int64_t j = toff[i]; j < toff[i + 1]; j++) tri_mesh[(size_t)j] = i;
        mt[i] = make_int2((int)tileoff[i], (int)tileoff[i + 1]);
    }
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->tri_mesh, tri_mesh.data(), sizeof(int32_t) * b->m, cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(b->mesh_tiles, mt.data(), sizeof(int2) * n, cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LSM_OK;
}

void batch_release(Batch* b)
{
    void* ps[] = {b->verts, b->tris, b->tri_sigma, b->vpn, b->tri_mesh, b->s32_pos, b->s32_nw, b->s32_lo,
                  b->s32_nwlo, b->s64_pos, b->s64_nw, b->tile_lo, b->tile_hi, b->tile_chi, b->tile_clo,
                  b->mesh_tiles};
    for (void* p : ps)
        if (p) cudaFree(p);
}

}  // namespace lsm
