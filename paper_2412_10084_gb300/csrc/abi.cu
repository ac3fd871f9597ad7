// C ABI of the ProbeSDF render library: handles, host-side validation,
// launch configuration, dense <-> packed grid conversion.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"
#include "probesdf.h"
#include "proposal.h"
#include "tc_sm100.cuh"

struct psdf_grid {
    psdf_grid_desc desc;
    const void* values;
};
struct psdf_probes {
    psdf_probe_desc desc;
    const void* coeffs;
};
struct psdf_mlp {
    psdf_mlp_desc desc;
    const void* params;
};

// Device status word (per device, static storage): kernels OR error bits into
// it; psdf_device_status reads and clears it.
__device__ int g_device_status;

namespace {

thread_local int32_t g_last_cuda_error = 0;
// Polls of each tensor-core completion wait in the kernels this thread launches.
thread_local uint32_t g_wait_polls = psdf::tc::kWaitPolls;

// Address of g_device_status on the current device (looked up once per device).
int* device_status_ptr()
{
    static int* ptrs[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
        ptrs[dev] = static_cast<int*>(p);
    }
    return ptrs[dev];
}

psdf_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return PSDF_OK;
    g_last_cuda_error = static_cast<int32_t>(e);
    return PSDF_ERR_CUDA;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

psdf_status check_grid_desc(const psdf_grid_desc* d)
{
    if (!d) return PSDF_ERR_INVALID_ARG;
    int64_t n = 1;
    for (int a = 0; a < 3; ++a) {
        if (d->dims[a] < 2 || d->dims[a] > 4096) return PSDF_ERR_BAD_SHAPE;
        if (!(d->box_max[a] > d->box_min[a])) return PSDF_ERR_BAD_SHAPE;
        n *= d->dims[a];
    }
    if (n >= (int64_t(1) << 31)) return PSDF_ERR_BAD_SHAPE;
    if (d->feat_dtype != PSDF_F32 && d->feat_dtype != PSDF_BF16) return PSDF_ERR_BAD_DTYPE;
    if (d->n_feat != 3) return PSDF_ERR_UNSUPPORTED;
    if (d->feat_layout != PSDF_FEAT_NODES && d->feat_layout != PSDF_FEAT_TRIPLANE)
        return PSDF_ERR_INVALID_ARG;
    if (d->feat_layout == PSDF_FEAT_TRIPLANE && d->feat_dtype != PSDF_F32)
        return PSDF_ERR_UNSUPPORTED;
    if (d->n_bricks < 0) return PSDF_ERR_INVALID_ARG;
    if (d->n_bricks > 0) {
        if (d->feat_layout != PSDF_FEAT_NODES || d->feat_dtype != PSDF_F32)
            return PSDF_ERR_UNSUPPORTED;
        for (int a = 0; a < 3; ++a)
            if (d->dims[a] % PSDF_TILE != 0) return PSDF_ERR_BAD_SHAPE;
        if (d->n_bricks > n / 4096) return PSDF_ERR_BAD_SHAPE;
        if (!std::isfinite(d->empty_sdf)) return PSDF_ERR_INVALID_ARG;
    }
    return PSDF_OK;
}

bool sparse(const psdf_grid_desc* d) { return d->n_bricks > 0; }

int64_t n_brick_cells(const psdf_grid_desc* d)
{
    return int64_t(d->dims[0] / PSDF_TILE) * (d->dims[1] / PSDF_TILE) * (d->dims[2] / PSDF_TILE);
}

// Bytes of the brick table (padded to 16).
size_t brick_table_bytes(const psdf_grid_desc* d)
{
    return (static_cast<size_t>(n_brick_cells(d)) * 4 + 15) & ~size_t(15);
}

int tri_tiles(int32_t dims) { return (dims - 1 + PSDF_TILE - 1) / PSDF_TILE; }

int64_t tri_texels(const psdf_grid_desc* d)
{
    return int64_t(tri_tiles(d->dims[0])) * tri_tiles(d->dims[1]) * tri_tiles(d->dims[2]) * 3 *
           PSDF_TILE * PSDF_TILE;
}

int64_t grid_nodes(const psdf_grid_desc* d)
{
    return int64_t(d->dims[0]) * d->dims[1] * d->dims[2];
}

// Byte offset of the BF16 feature records in the BF16-feature layout.
size_t bf16_feat_offset(const psdf_grid_desc* d)
{
    return (static_cast<size_t>(grid_nodes(d)) * 4 + 15) & ~size_t(15);
}

// Device pointers of a grid's packed values (the layouts of psdf_grid_bytes).
void set_grid_view(const psdf_grid_desc& gd, const void* values, psdf::GridView& g)
{
    const uint8_t* base = static_cast<const uint8_t*>(values);
    if (sparse(&gd)) {
        g.table = reinterpret_cast<const int*>(base);
        g.nodes = reinterpret_cast<const float4*>(base + brick_table_bytes(&gd));
        for (int a = 0; a < 3; ++a) g.B[a] = gd.dims[a] / PSDF_TILE;
        g.empty_sdf = gd.empty_sdf;
        g.n_bricks = gd.n_bricks;
        g.rec_off = static_cast<int64_t>(brick_table_bytes(&gd) / 4);
    } else if (gd.feat_layout == PSDF_FEAT_TRIPLANE) {
        g.sdf = reinterpret_cast<const float*>(base);
        g.planes = reinterpret_cast<const float4*>(base + bf16_feat_offset(&gd));
        g.plane_off = static_cast<int64_t>(bf16_feat_offset(&gd) / 4);
        for (int a = 0; a < 3; ++a) g.tiles[a] = tri_tiles(gd.dims[a]);
    } else if (gd.feat_dtype == PSDF_BF16) {
        g.sdf = reinterpret_cast<const float*>(base);
        g.feat16 = reinterpret_cast<const uint2*>(base + bf16_feat_offset(&gd));
    } else {
        g.nodes = static_cast<const float4*>(values);
    }
}

psdf_status check_probe_desc(const psdf_probe_desc* d)
{
    if (!d) return PSDF_ERR_INVALID_ARG;
    int64_t n = 1;
    for (int a = 0; a < 3; ++a) {
        if (d->dims[a] < 2 || d->dims[a] > 4096) return PSDF_ERR_BAD_SHAPE;
        n *= d->dims[a];
    }
    if (d->sh_l < 1 || d->sh_l > 4 || d->n_ang < 1 || d->n_ang > 64) return PSDF_ERR_BAD_SHAPE;
    if (n * d->sh_l * d->sh_l * d->n_ang >= (int64_t(1) << 31)) return PSDF_ERR_BAD_SHAPE;
    if (d->dtype != PSDF_F32 && d->dtype != PSDF_F16) return PSDF_ERR_BAD_DTYPE;
    if (d->dtype == PSDF_F16 && d->n_ang % 4 != 0) return PSDF_ERR_UNSUPPORTED;
    return PSDF_OK;
}

psdf_status check_mlp_desc(const psdf_mlp_desc* d)
{
    if (!d) return PSDF_ERR_INVALID_ARG;
    if (d->n_in < 1 || d->n_in > 64 || d->width < 1 || d->width > 256) return PSDF_ERR_BAD_SHAPE;
    if (d->dtype != PSDF_F32 && d->dtype != PSDF_F16) return PSDF_ERR_BAD_DTYPE;
    return PSDF_OK;
}

int64_t mlp_params(const psdf_mlp_desc* d)
{
    const int64_t W = d->width, n = d->n_in;
    return W * n + W + W * W + W + 3 * W + 3;
}

struct Resolved {
    psdf::RenderArgs args;
    psdf::KernelShape shape;
};

psdf_status resolve(const psdf_grid* grid, const psdf_probes* probes, const psdf_mlp* mlp,
                    const psdf_render_params* p, const float* rays_o, const float* rays_d,
                    const float* t_samples, int64_t n_rays, Resolved& r)
{
    if (!grid || !probes || !mlp || !p) return PSDF_ERR_INVALID_ARG;
    if (n_rays < 0) return PSDF_ERR_INVALID_ARG;
    if (n_rays > 0 && (!rays_o || !rays_d)) return PSDF_ERR_INVALID_ARG;
    if (!(p->tau > 0.0f) || p->n_samples < 1 || p->n_samples > 4096) return PSDF_ERR_BAD_SHAPE;
    if (p->dir_mode != PSDF_DIR_REFLECT && p->dir_mode != PSDF_DIR_VIEW)
        return PSDF_ERR_INVALID_ARG;
    if (p->n_fresnel < 0 || p->n_fresnel > 8) return PSDF_ERR_BAD_SHAPE;
    if (p->n_bins < 0 || p->n_bins > 32) return PSDF_ERR_BAD_SHAPE;
    if (p->n_bins > 0 && n_rays > 0 && !t_samples) return PSDF_ERR_INVALID_ARG;
    const psdf_grid_desc& gd = grid->desc;
    const psdf_probe_desc& pd = probes->desc;
    const psdf_mlp_desc& md = mlp->desc;
    if (md.n_in != gd.n_feat + pd.n_ang + p->n_fresnel) return PSDF_ERR_BAD_SHAPE;
    if (!grid->values || !probes->coeffs || !mlp->params) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(grid->values) || !aligned16(probes->coeffs) || !aligned16(mlp->params))
        return PSDF_ERR_MISALIGNED;
    if (!aligned16(rays_o) || !aligned16(rays_d) || !aligned16(t_samples))
        return PSDF_ERR_MISALIGNED;
    r.shape.na = pd.n_ang;
    r.shape.l2 = pd.sh_l * pd.sh_l;
    r.shape.width = md.width;
    r.shape.k = p->n_fresnel;
    r.shape.fb = sparse(&gd) ? 3
                 : gd.feat_layout == PSDF_FEAT_TRIPLANE ? 2
                                                         : (gd.feat_dtype == PSDF_BF16 ? 1 : 0);
    r.shape.ph = pd.dtype == PSDF_F16;
    r.shape.mh = md.dtype == PSDF_F16;
    bool known = false;
#define PSDF_KNOWN(NA, L2, W, K, FB, PH, MH) \
    if (r.shape.match(NA, L2, W, K, FB, PH, MH)) known = true;
    PSDF_FOR_EACH_SHAPE(PSDF_KNOWN)
#undef PSDF_KNOWN
    if (!known) return PSDF_ERR_UNSUPPORTED;

    psdf::RenderArgs& A = r.args;
    std::memset(&A, 0, sizeof(A));
    set_grid_view(gd, grid->values, A.grid);
    for (int a = 0; a < 3; ++a) {
        A.grid.R[a] = gd.dims[a];
        A.grid.bmin[a] = gd.box_min[a];
        A.grid.bmax[a] = gd.box_max[a];
        // (R - 1) / (bmax - bmin) in FP32; the sample positions depend on these bits
        const volatile float ext = gd.box_max[a] - gd.box_min[a];
        A.grid.sc[a] = static_cast<float>(gd.dims[a] - 1) / ext;
        A.probes.P[a] = pd.dims[a];
        A.probes.sc[a] = static_cast<float>(pd.dims[a] - 1) / ext;
    }
    if (r.shape.ph)
        A.probes.coeffs16 = static_cast<const uint2*>(probes->coeffs);
    else
        A.probes.coeffs = static_cast<const float4*>(probes->coeffs);
    A.mlp = static_cast<const float*>(mlp->params);
    A.tau = p->tau;
    A.n_samples = p->n_samples;
    A.dir_mode = p->dir_mode;
    for (int c = 0; c < 3; ++c) A.bg[c] = p->bg[c];
    A.rays_o = rays_o;
    A.rays_d = rays_d;
    A.t_samples = t_samples;
    A.n_bins = t_samples ? p->n_bins : 0;
    A.n_rays = n_rays;
    A.status = device_status_ptr();
    A.wait_polls = g_wait_polls;
    if (!A.status) return cuda_status(cudaErrorInvalidDevice);
    return PSDF_OK;
}

// Persistent-grid size: every SM filled to its occupancy, capped by the work.
int grid_size(int64_t n_rays, int ctas_per_sm, int warps_per_cta)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    if (ctas_per_sm <= 0) ctas_per_sm = 1;
    const int64_t full = int64_t(sms) * ctas_per_sm;
    const int64_t need = (n_rays + warps_per_cta - 1) / warps_per_cta;
    return static_cast<int>(need < full ? need : full);
}

__global__ void pack_kernel(const float* __restrict__ sdf, const float* __restrict__ feat,
                            float4* __restrict__ out, int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = make_float4(sdf[i], feat[3 * i], feat[3 * i + 1], feat[3 * i + 2]);
}

__global__ void unpack_kernel(const float4* __restrict__ in, float* __restrict__ sdf,
                              float* __restrict__ feat, int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float4 v = in[i];
        if (sdf) sdf[i] = v.x;
        if (feat) {
            feat[3 * i] = v.y;
            feat[3 * i + 1] = v.z;
            feat[3 * i + 2] = v.w;
        }
    }
}

// Sparse bricks: dense SDF and features [R^3][3] <-> the stored bricks' node
// records (the table in front of them says which).  Unpack fills the nodes of
// bricks that are not stored with {fill, 0, 0, 0}.
__global__ void brick_copy_kernel(int Rx, int Ry, int Rz, const int* __restrict__ table,
                                  int n_bricks, float4* __restrict__ bricks,
                                  float* __restrict__ sdf, float* __restrict__ feat, float fill,
                                  bool pack)
{
    const int64_t n = int64_t(Rx) * Ry * Rz;
    const int Bx = Rx / 16, By = Ry / 16;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % Rx), y = static_cast<int>((i / Rx) % Ry);
        const int z = static_cast<int>(i / (int64_t(Rx) * Ry));
        int slot = table[((z >> 4) * By + (y >> 4)) * Bx + (x >> 4)];
        if (slot >= n_bricks) slot = -1;  // a table entry out of range stores nothing
        const int64_t rec = int64_t(slot) * 4096 + (((z & 15) * 16 + (y & 15)) * 16 + (x & 15));
        if (pack) {
            if (slot >= 0)
                bricks[rec] = make_float4(sdf[i], feat[3 * i], feat[3 * i + 1], feat[3 * i + 2]);
        } else {
            const float4 v = slot >= 0 ? bricks[rec] : make_float4(fill, 0.f, 0.f, 0.f);
            if (sdf) sdf[i] = v.x;
            if (feat) {
                feat[3 * i] = v.y;
                feat[3 * i + 1] = v.z;
                feat[3 * i + 2] = v.w;
            }
        }
    }
}

// Tri-plane layout: dense SDF and planes [..][3] <-> the packed SDF array and
// 16-byte texels (either dense pointer may be null).
__global__ void tri_copy_kernel(float* __restrict__ sdf, float* __restrict__ planes,
                                float* __restrict__ out_sdf, float4* __restrict__ out_tex,
                                int64_t n_nodes, int64_t n_texels, bool pack)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
         i < (n_nodes > n_texels ? n_nodes : n_texels); i += int64_t(gridDim.x) * blockDim.x) {
        if (i < n_nodes && sdf) {
            if (pack)
                out_sdf[i] = sdf[i];
            else
                sdf[i] = out_sdf[i];
        }
        if (i < n_texels && planes) {
            if (pack) {
                out_tex[i] = make_float4(planes[3 * i], planes[3 * i + 1], planes[3 * i + 2], 0.f);
            } else {
                const float4 v = out_tex[i];
                planes[3 * i] = v.x;
                planes[3 * i + 1] = v.y;
                planes[3 * i + 2] = v.z;
            }
        }
    }
}

__device__ __forceinline__ uint32_t bf16_bits(float v)
{
    // round to nearest even; NaN stays NaN
    const uint32_t u = __float_as_uint(v);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (u >> 16) | 0x40u;
    return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}

__global__ void pack_bf16_kernel(const float* __restrict__ sdf, const float* __restrict__ feat,
                                 float* __restrict__ out_sdf, uint2* __restrict__ out_feat,
                                 int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        out_sdf[i] = sdf[i];
        const uint32_t f0 = bf16_bits(feat[3 * i]), f1 = bf16_bits(feat[3 * i + 1]);
        const uint32_t f2 = bf16_bits(feat[3 * i + 2]);
        out_feat[i] = make_uint2(f0 | (f1 << 16), f2);
    }
}

__global__ void unpack_bf16_kernel(const float* __restrict__ in_sdf,
                                   const uint2* __restrict__ in_feat, float* __restrict__ sdf,
                                   float* __restrict__ feat, int64_t n)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        if (sdf) sdf[i] = in_sdf[i];
        if (feat) {
            const uint2 f = in_feat[i];
            feat[3 * i] = __uint_as_float(f.x << 16);
            feat[3 * i + 1] = __uint_as_float(f.x & 0xffff0000u);
            feat[3 * i + 2] = __uint_as_float(f.y << 16);
        }
    }
}

}  // namespace

namespace psdf {

int resident_ctas(const cudaFuncAttributes& fa, int threads, size_t dyn_smem, unsigned tmem_cols)
{
    int dev = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0, blk_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int warps = (threads + 31) / 32;
    // registers are allocated per warp in units of 256
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int n = blk_sm > 0 ? blk_sm : 32;
    if (regs_warp > 0) n = std::min(n, regs_sm / (regs_warp * warps));
    const size_t smem = dyn_smem + fa.sharedSizeBytes + static_cast<size_t>(reserved);
    if (smem > 0) n = std::min<int>(n, static_cast<int>(smem_sm / smem));
    n = std::min(n, thr_sm / threads);
    if (tmem_cols > 0) n = std::min<int>(n, static_cast<int>(512 / tmem_cols));
    return n;
}

cudaError_t set_smem_carveout(const void* func, int threads, size_t dyn_smem, unsigned tmem_cols)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    const int n = resident_ctas(fa, threads, dyn_smem, tmem_cols);
    int dev = 0, smem_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (n <= 0 || smem_sm <= 0) return cudaSuccess;  // nothing to choose
    const size_t need =
        static_cast<size_t>(n) * (dyn_smem + fa.sharedSizeBytes + static_cast<size_t>(reserved));
    // The shared-memory capacities an sm_100-family SM can be split into
    // (KiB); the hint is a percentage of the largest, rounded up by the driver
    // to the next capacity, so the smallest one that holds `need` is asked for
    // just below its own value.
    static const int kCapKiB[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
    int pct = 100;
    for (int c : kCapKiB) {
        const size_t cap = static_cast<size_t>(c) * 1024;
        if (cap >= need && cap <= static_cast<size_t>(smem_sm)) {
            pct = static_cast<int>((100 * cap) / static_cast<size_t>(smem_sm));
            break;
        }
    }
    return cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

cudaError_t launch_pack(const float* sdf, const float* feat, float4* packed, int64_t n_nodes,
                        cudaStream_t stream)
{
    const int threads = 256;
    const int64_t blocks = (n_nodes + threads - 1) / threads;
    pack_kernel<<<(int)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0, stream>>>(
        sdf, feat, packed, n_nodes);
    return cudaGetLastError();
}

cudaError_t launch_pack_bf16(const float* sdf, const float* feat, void* packed, size_t feat_off,
                             int64_t n_nodes, cudaStream_t stream)
{
    const int threads = 256;
    const int64_t blocks = (n_nodes + threads - 1) / threads;
    uint8_t* base = static_cast<uint8_t*>(packed);
    pack_bf16_kernel<<<(int)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0, stream>>>(
        sdf, feat, reinterpret_cast<float*>(base), reinterpret_cast<uint2*>(base + feat_off),
        n_nodes);
    return cudaGetLastError();
}

cudaError_t launch_unpack_bf16(const void* packed, size_t feat_off, float* sdf, float* feat,
                               int64_t n_nodes, cudaStream_t stream)
{
    const int threads = 256;
    const int64_t blocks = (n_nodes + threads - 1) / threads;
    const uint8_t* base = static_cast<const uint8_t*>(packed);
    unpack_bf16_kernel<<<(int)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0,
                         stream>>>(reinterpret_cast<const float*>(base),
                                   reinterpret_cast<const uint2*>(base + feat_off), sdf, feat,
                                   n_nodes);
    return cudaGetLastError();
}

cudaError_t launch_brick_copy(const int dims[3], int n_bricks, const int* table, float4* bricks,
                              float* sdf, float* feat, float fill, bool pack,
                              cudaStream_t stream)
{
    const int threads = 256;
    const int64_t n = int64_t(dims[0]) * dims[1] * dims[2];
    const int64_t blocks = (n + threads - 1) / threads;
    brick_copy_kernel<<<(int)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0, stream>>>(
        dims[0], dims[1], dims[2], table, n_bricks, bricks, sdf, feat, fill, pack);
    return cudaGetLastError();
}

cudaError_t launch_tri_copy(const float* sdf, const float* planes, void* packed, size_t plane_off,
                            int64_t n_nodes, int64_t n_texels, bool pack, cudaStream_t stream)
{
    const int threads = 256;
    const int64_t n = n_nodes > n_texels ? n_nodes : n_texels;
    const int64_t blocks = (n + threads - 1) / threads;
    uint8_t* base = static_cast<uint8_t*>(packed);
    tri_copy_kernel<<<(int)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0, stream>>>(
        const_cast<float*>(sdf), const_cast<float*>(planes), reinterpret_cast<float*>(base),
        reinterpret_cast<float4*>(base + plane_off), n_nodes, n_texels, pack);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const float4* packed, float* sdf, float* feat, int64_t n_nodes,
                          cudaStream_t stream)
{
    const int threads = 256;
    const int64_t blocks = (n_nodes + threads - 1) / threads;
    unpack_kernel<<<(int)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0, stream>>>(
        packed, sdf, feat, n_nodes);
    return cudaGetLastError();
}

}  // namespace psdf

extern "C" {

const char* psdf_status_string(psdf_status s)
{
    switch (s) {
        case PSDF_OK: return "ok";
        case PSDF_ERR_INVALID_ARG: return "invalid argument";
        case PSDF_ERR_BAD_SHAPE: return "shape outside the supported range";
        case PSDF_ERR_BAD_DTYPE: return "unsupported dtype";
        case PSDF_ERR_MISALIGNED: return "device pointer not 16-byte aligned";
        case PSDF_ERR_CUDA: return "CUDA error";
        case PSDF_ERR_UNSUPPORTED: return "combination not compiled in";
        default: return "unknown status";
    }
}

int32_t psdf_last_cuda_error(void) { return g_last_cuda_error; }

int32_t psdf_version(void) { return 200; }

psdf_status psdf_set_wait_polls(uint32_t polls)
{
    g_wait_polls = polls == 0xFFFFFFFFu ? psdf::tc::kWaitPolls : polls;
    return PSDF_OK;
}

uint32_t psdf_wait_polls(void) { return g_wait_polls; }

psdf_status psdf_device_status(void* stream, int32_t* flags)
{
    if (!flags) return PSDF_ERR_INVALID_ARG;
    int* p = device_status_ptr();
    if (!p) return cuda_status(cudaErrorInvalidDevice);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, p, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    *flags = v;
    return PSDF_OK;
}

psdf_status psdf_grid_bytes(const psdf_grid_desc* desc, size_t* values_bytes, size_t* grad_bytes)
{
    const psdf_status st = check_grid_desc(desc);
    if (st != PSDF_OK) return st;
    if (!values_bytes || !grad_bytes) return PSDF_ERR_INVALID_ARG;
    const size_t n = static_cast<size_t>(grid_nodes(desc));
    if (sparse(desc)) {
        *values_bytes = *grad_bytes =
            brick_table_bytes(desc) + 16 * 4096 * static_cast<size_t>(desc->n_bricks);
        return PSDF_OK;
    }
    if (desc->feat_layout == PSDF_FEAT_TRIPLANE) {
        *values_bytes = *grad_bytes = bf16_feat_offset(desc) + 16 * size_t(tri_texels(desc));
        return PSDF_OK;
    }
    *values_bytes = desc->feat_dtype == PSDF_BF16 ? bf16_feat_offset(desc) + 8 * n : 16 * n;
    *grad_bytes = 16 * n;
    return PSDF_OK;
}

psdf_status psdf_grid_create(const psdf_grid_desc* desc, const void* values, psdf_grid** out)
{
    const psdf_status st = check_grid_desc(desc);
    if (st != PSDF_OK) return st;
    if (!values || !out) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(values)) return PSDF_ERR_MISALIGNED;
    psdf_grid* g = new (std::nothrow) psdf_grid;
    if (!g) return PSDF_ERR_INVALID_ARG;
    g->desc = *desc;
    g->values = values;
    *out = g;
    return PSDF_OK;
}

void psdf_grid_destroy(psdf_grid* grid) { delete grid; }

psdf_status psdf_grid_pack(const psdf_grid_desc* desc, const float* sdf, const float* feat,
                           void* packed, void* stream)
{
    const psdf_status st = check_grid_desc(desc);
    if (st != PSDF_OK) return st;
    if (!sdf || !feat || !packed) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(packed)) return PSDF_ERR_MISALIGNED;
    const int64_t n = grid_nodes(desc);
    if (sparse(desc))
        return cuda_status(psdf::launch_brick_copy(
            desc->dims, desc->n_bricks, static_cast<const int*>(packed),
            reinterpret_cast<float4*>(static_cast<uint8_t*>(packed) + brick_table_bytes(desc)),
            const_cast<float*>(sdf), const_cast<float*>(feat), 0.0f, true,
            static_cast<cudaStream_t>(stream)));
    if (desc->feat_layout == PSDF_FEAT_TRIPLANE)
        return cuda_status(psdf::launch_tri_copy(sdf, feat, packed, bf16_feat_offset(desc), n,
                                                 tri_texels(desc), true,
                                                 static_cast<cudaStream_t>(stream)));
    if (desc->feat_dtype == PSDF_BF16)
        return cuda_status(psdf::launch_pack_bf16(sdf, feat, packed, bf16_feat_offset(desc), n,
                                                  static_cast<cudaStream_t>(stream)));
    return cuda_status(psdf::launch_pack(sdf, feat, static_cast<float4*>(packed), n,
                                         static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_grid_unpack(const psdf_grid_desc* desc, int32_t which, const void* packed,
                             float* sdf, float* feat, void* stream)
{
    const psdf_status st = check_grid_desc(desc);
    if (st != PSDF_OK) return st;
    if (!packed || (!sdf && !feat)) return PSDF_ERR_INVALID_ARG;
    if (which != PSDF_GRID_VALUES && which != PSDF_GRID_GRAD) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(packed)) return PSDF_ERR_MISALIGNED;
    const int64_t n = grid_nodes(desc);
    if (sparse(desc))
        return cuda_status(psdf::launch_brick_copy(
            desc->dims, desc->n_bricks, static_cast<const int*>(packed),
            reinterpret_cast<float4*>(const_cast<uint8_t*>(static_cast<const uint8_t*>(packed)) +
                                      brick_table_bytes(desc)),
            sdf, feat, which == PSDF_GRID_VALUES ? desc->empty_sdf : 0.0f, false,
            static_cast<cudaStream_t>(stream)));
    if (desc->feat_layout == PSDF_FEAT_TRIPLANE)
        return cuda_status(psdf::launch_tri_copy(sdf, feat, const_cast<void*>(packed),
                                                 bf16_feat_offset(desc), n, tri_texels(desc),
                                                 false, static_cast<cudaStream_t>(stream)));
    if (which == PSDF_GRID_VALUES && desc->feat_dtype == PSDF_BF16)
        return cuda_status(psdf::launch_unpack_bf16(packed, bf16_feat_offset(desc), sdf, feat, n,
                                                    static_cast<cudaStream_t>(stream)));
    return cuda_status(psdf::launch_unpack(static_cast<const float4*>(packed), sdf, feat, n,
                                           static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_probes_create(const psdf_probe_desc* desc, const void* coeffs,
                               psdf_probes** out)
{
    const psdf_status st = check_probe_desc(desc);
    if (st != PSDF_OK) return st;
    if (!coeffs || !out) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(coeffs)) return PSDF_ERR_MISALIGNED;
    psdf_probes* p = new (std::nothrow) psdf_probes;
    if (!p) return PSDF_ERR_INVALID_ARG;
    p->desc = *desc;
    p->coeffs = coeffs;
    *out = p;
    return PSDF_OK;
}

void psdf_probes_destroy(psdf_probes* probes) { delete probes; }

psdf_status psdf_mlp_param_count(const psdf_mlp_desc* desc, int64_t* count)
{
    const psdf_status st = check_mlp_desc(desc);
    if (st != PSDF_OK) return st;
    if (!count) return PSDF_ERR_INVALID_ARG;
    *count = mlp_params(desc);
    return PSDF_OK;
}

psdf_status psdf_mlp_create(const psdf_mlp_desc* desc, const void* params, psdf_mlp** out)
{
    const psdf_status st = check_mlp_desc(desc);
    if (st != PSDF_OK) return st;
    if (!params || !out) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(params)) return PSDF_ERR_MISALIGNED;
    psdf_mlp* m = new (std::nothrow) psdf_mlp;
    if (!m) return PSDF_ERR_INVALID_ARG;
    m->desc = *desc;
    m->params = params;
    *out = m;
    return PSDF_OK;
}

void psdf_mlp_destroy(psdf_mlp* mlp) { delete mlp; }

psdf_status psdf_render_forward(const psdf_grid* grid, const psdf_probes* probes,
                                const psdf_mlp* mlp, const psdf_render_params* params,
                                const float* rays_o, const float* rays_d,
                                const float* t_samples, int64_t n_rays, float* rgb,
                                float* depth, float* wsum, float* logT_final, int32_t* n_live,
                                void* stream)
{
    Resolved r;
    psdf_status st = resolve(grid, probes, mlp, params, rays_o, rays_d, t_samples, n_rays, r);
    if (st != PSDF_OK) return st;
    if (n_rays > 0 && (!rgb || !depth || !wsum || !logT_final)) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(rgb) || !aligned16(depth) || !aligned16(wsum) || !aligned16(logT_final) ||
        !aligned16(n_live))
        return PSDF_ERR_MISALIGNED;
    if (n_rays == 0) return PSDF_OK;
    r.args.rgb = rgb;
    r.args.depth = depth;
    r.args.wsum = wsum;
    r.args.logT = logT_final;
    r.args.n_live = n_live;
    int per_sm = 0;
    st = cuda_status(psdf::forward_ctas_per_sm(r.shape, &per_sm));
    if (st != PSDF_OK) return st;
    const int ctas = grid_size(n_rays, per_sm, psdf::kFwdThreads / 32);
    return cuda_status(
        psdf::launch_forward(r.args, r.shape, ctas, static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_render_backward(const psdf_grid* grid, const psdf_probes* probes,
                                 const psdf_mlp* mlp, const psdf_render_params* params,
                                 const float* rays_o, const float* rays_d,
                                 const float* t_samples, int64_t n_rays, const float* d_rgb,
                                 const float* d_depth, const float* d_wsum,
                                 const float* logT_final, const int32_t* n_live,
                                 float* grad_grid, float* grad_probes, float* grad_mlp,
                                 void* stream)
{
    Resolved r;
    psdf_status st = resolve(grid, probes, mlp, params, rays_o, rays_d, t_samples, n_rays, r);
    if (st != PSDF_OK) return st;
    if (!grad_grid || !grad_probes || !grad_mlp) return PSDF_ERR_INVALID_ARG;
    if (n_rays > 0 && (!d_rgb || !logT_final)) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(d_rgb) || !aligned16(d_depth) || !aligned16(d_wsum) ||
        !aligned16(logT_final) || !aligned16(n_live) || !aligned16(grad_grid) ||
        !aligned16(grad_probes) || !aligned16(grad_mlp))
        return PSDF_ERR_MISALIGNED;
    if (n_rays == 0) return PSDF_OK;
    r.args.logT = const_cast<float*>(logT_final);
    r.args.n_live = const_cast<int32_t*>(n_live);
    r.args.d_rgb = d_rgb;
    r.args.d_depth = d_depth;
    r.args.d_wsum = d_wsum;
    r.args.grad_grid = grad_grid;
    r.args.grad_probes = grad_probes;
    r.args.grad_mlp = grad_mlp;
    int per_sm = 0;
    st = cuda_status(psdf::backward_ctas_per_sm(r.shape, &per_sm));
    if (st != PSDF_OK) return st;
    const int ctas = grid_size(n_rays, per_sm, psdf::kBwdThreads / 32);
    return cuda_status(
        psdf::launch_backward(r.args, r.shape, ctas, static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_render_occupancy(const psdf_grid* grid, const psdf_probes* probes,
                                  const psdf_mlp* mlp, const psdf_render_params* params,
                                  int32_t* forward_ctas_per_sm, int32_t* backward_ctas_per_sm)
{
    Resolved r;
    psdf_status st = resolve(grid, probes, mlp, params, nullptr, nullptr, nullptr, 0, r);
    if (st != PSDF_OK) return st;
    if (!forward_ctas_per_sm || !backward_ctas_per_sm) return PSDF_ERR_INVALID_ARG;
    int f = 0, b = 0;
    st = cuda_status(psdf::forward_ctas_per_sm(r.shape, &f));
    if (st != PSDF_OK) return st;
    st = cuda_status(psdf::backward_ctas_per_sm(r.shape, &b));
    if (st != PSDF_OK) return st;
    *forward_ctas_per_sm = f;
    *backward_ctas_per_sm = b;
    return PSDF_OK;
}


// ---------------------------------------------------------------------------
// Optimiser
// ---------------------------------------------------------------------------

psdf_status psdf_adam_step(float* param, float* grad, float* m, float* v, int64_t n, float lr,
                           float beta1, float beta2, float eps, int32_t step, int32_t clear_grad,
                           void* stream)
{
    if (n < 0 || step < 1) return PSDF_ERR_INVALID_ARG;
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        return PSDF_ERR_INVALID_ARG;
    if (n == 0) return PSDF_OK;
    if (!param || !grad || !m || !v) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(param) || !aligned16(grad) || !aligned16(m) || !aligned16(v))
        return PSDF_ERR_MISALIGNED;
    return cuda_status(psdf::launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, step,
                                         clear_grad, static_cast<cudaStream_t>(stream)));
}

// ---------------------------------------------------------------------------
// Two-pass inference
// ---------------------------------------------------------------------------

psdf_status psdf_colour_field_bytes(const psdf_grid_desc* desc, size_t* bytes)
{
    const psdf_status st = check_grid_desc(desc);
    if (st != PSDF_OK) return st;
    if (!bytes) return PSDF_ERR_INVALID_ARG;
    *bytes = 8 * static_cast<size_t>(grid_nodes(desc));
    return PSDF_OK;
}

psdf_status psdf_shade_nodes(const psdf_grid* grid, const psdf_probes* probes,
                             const psdf_mlp* mlp, const psdf_render_params* params,
                             const float camera[3], float band, void* colours, void* stream)
{
    Resolved r;
    psdf_status st = resolve(grid, probes, mlp, params, nullptr, nullptr, nullptr, 0, r);
    if (st != PSDF_OK) return st;
    if (!camera || !colours || !(band >= 0.0f)) return PSDF_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(camera[a])) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(colours)) return PSDF_ERR_MISALIGNED;
    psdf::ShadeArgs S;
    const psdf_grid_desc& gd = grid->desc;
    for (int a = 0; a < 3; ++a) {
        S.cam[a] = camera[a];
        S.h[a] = (gd.box_max[a] - gd.box_min[a]) / static_cast<float>(gd.dims[a] - 1);
    }
    S.band = band;
    S.colours = static_cast<uint2*>(colours);
    return cuda_status(
        psdf::launch_shade(r.args, r.shape, S, static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_render_colour_field(const psdf_grid* grid, const void* colours,
                                     const psdf_render_params* p, const float* rays_o,
                                     const float* rays_d, const float* t_samples,
                                     int64_t n_rays, float* rgb, float* depth, float* wsum,
                                     void* stream)
{
    if (!grid || !grid->values || !p || !colours) return PSDF_ERR_INVALID_ARG;
    if (n_rays < 0) return PSDF_ERR_INVALID_ARG;
    if (!(p->tau > 0.0f) || p->n_samples < 1 || p->n_samples > 4096) return PSDF_ERR_BAD_SHAPE;
    if (p->n_bins < 0 || p->n_bins > 32) return PSDF_ERR_BAD_SHAPE;
    if (n_rays > 0 && (!rays_o || !rays_d || !rgb || !depth || !wsum))
        return PSDF_ERR_INVALID_ARG;
    if (p->n_bins > 0 && n_rays > 0 && !t_samples) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(grid->values) || !aligned16(colours) || !aligned16(rays_o) ||
        !aligned16(rays_d) || !aligned16(t_samples) || !aligned16(rgb) || !aligned16(depth) ||
        !aligned16(wsum))
        return PSDF_ERR_MISALIGNED;
    if (n_rays == 0) return PSDF_OK;
    psdf::RenderArgs A;
    std::memset(&A, 0, sizeof(A));
    const psdf_grid_desc& gd = grid->desc;
    set_grid_view(gd, grid->values, A.grid);
    for (int a = 0; a < 3; ++a) {
        A.grid.R[a] = gd.dims[a];
        A.grid.bmin[a] = gd.box_min[a];
        A.grid.bmax[a] = gd.box_max[a];
        // the same FP32 scale as the per-sample render, so samples land on the same cells
        const volatile float ext = gd.box_max[a] - gd.box_min[a];
        A.grid.sc[a] = static_cast<float>(gd.dims[a] - 1) / ext;
    }
    A.tau = p->tau;
    A.n_samples = p->n_samples;
    for (int c = 0; c < 3; ++c) A.bg[c] = p->bg[c];
    A.rays_o = rays_o;
    A.rays_d = rays_d;
    A.t_samples = t_samples;
    A.n_bins = t_samples ? p->n_bins : 0;
    A.n_rays = n_rays;
    A.rgb = rgb;
    A.depth = depth;
    A.wsum = wsum;
    return cuda_status(
        psdf::launch_colour_render(A, colours, static_cast<cudaStream_t>(stream)));
}

// ---------------------------------------------------------------------------
// Grid-level training terms
// ---------------------------------------------------------------------------

namespace {

// Element stride of the SDF slot in packed values / in a gradient buffer.
int sdf_value_stride(const psdf_grid_desc* d)
{
    return (d->feat_layout == PSDF_FEAT_NODES && d->feat_dtype == PSDF_F32) ? 4 : 1;
}

int sdf_grad_stride(const psdf_grid_desc* d)
{
    return d->feat_layout == PSDF_FEAT_NODES ? 4 : 1;
}

}  // namespace

psdf_status psdf_sdf_smooth(const psdf_grid_desc* desc, const float* sdf_hat, void* packed_values,
                            void* stream)
{
    const psdf_status st = check_grid_desc(desc);
    if (st != PSDF_OK) return st;
    if (!sdf_hat || !packed_values) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(sdf_hat) || !aligned16(packed_values)) return PSDF_ERR_MISALIGNED;
    if (sparse(desc))  // table, then {sdf, f0, f1, f2} records
        return cuda_status(psdf::launch_smooth_sparse(
            desc->dims, static_cast<const int*>(packed_values), desc->n_bricks, sdf_hat, 0, 1,
            static_cast<float*>(packed_values), static_cast<int64_t>(brick_table_bytes(desc) / 4),
            4, desc->empty_sdf, false, false, static_cast<cudaStream_t>(stream)));
    return cuda_status(psdf::launch_smooth(desc->dims, sdf_hat, 1,
                                           static_cast<float*>(packed_values),
                                           sdf_value_stride(desc), false, false,
                                           static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_sdf_smooth_adjoint(const psdf_grid_desc* desc, const void* grad_grid,
                                    float* d_sdf_hat, int32_t accumulate, void* stream)
{
    const psdf_status st = check_grid_desc(desc);
    if (st != PSDF_OK) return st;
    if (!grad_grid || !d_sdf_hat) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(grad_grid) || !aligned16(d_sdf_hat)) return PSDF_ERR_MISALIGNED;
    if (sparse(desc))  // the gradient buffer's copy of the table, then its records
        return cuda_status(psdf::launch_smooth_sparse(
            desc->dims, static_cast<const int*>(grad_grid), desc->n_bricks,
            static_cast<const float*>(grad_grid),
            static_cast<int64_t>(brick_table_bytes(desc) / 4), 4, d_sdf_hat, 0, 1, 0.0f, true,
            accumulate != 0, static_cast<cudaStream_t>(stream)));
    return cuda_status(psdf::launch_smooth(desc->dims, static_cast<const float*>(grad_grid),
                                           sdf_grad_stride(desc), d_sdf_hat, 1, true,
                                           accumulate != 0, static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_grid_regularizers(const psdf_grid_desc* desc, const float* sdf_hat,
                                   const void* packed_values, float lam_sdf, float lam_eik,
                                   float lam_normal, float lam_features, void* grad_grid,
                                   float* d_sdf_hat, float* loss, void* stream)
{
    const psdf_status st = check_grid_desc(desc);
    if (st != PSDF_OK) return st;
    if (!sdf_hat || !packed_values || !grad_grid || !d_sdf_hat) return PSDF_ERR_INVALID_ARG;
    if (!(lam_sdf >= 0.0f) || !(lam_eik >= 0.0f) || !(lam_normal >= 0.0f) ||
        !(lam_features >= 0.0f))
        return PSDF_ERR_INVALID_ARG;
    if (lam_features > 0.0f && desc->feat_layout != PSDF_FEAT_TRIPLANE)
        return PSDF_ERR_UNSUPPORTED;
    if (!aligned16(sdf_hat) || !aligned16(packed_values) || !aligned16(grad_grid) ||
        !aligned16(d_sdf_hat) || (loss && (reinterpret_cast<uintptr_t>(loss) & 3u)))
        return PSDF_ERR_MISALIGNED;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    float h[3];
    for (int a = 0; a < 3; ++a)
        h[a] = (desc->box_max[a] - desc->box_min[a]) / static_cast<float>(desc->dims[a] - 1);
    if (sparse(desc)) {  // the values' table, then {sdf, f0, f1, f2} records (and in the gradient)
        const int64_t rec = static_cast<int64_t>(brick_table_bytes(desc) / 4);
        return cuda_status(psdf::launch_sdf_reg(
            desc->dims, h, sdf_hat, static_cast<const float*>(packed_values) + rec, 4, lam_sdf,
            lam_eik, lam_normal, static_cast<float*>(grad_grid) + rec, 4, d_sdf_hat, loss, s,
            static_cast<const int*>(packed_values), desc->n_bricks, desc->empty_sdf));
    }
    cudaError_t e = psdf::launch_sdf_reg(
        desc->dims, h, sdf_hat, static_cast<const float*>(packed_values), sdf_value_stride(desc),
        lam_sdf, lam_eik, lam_normal, static_cast<float*>(grad_grid), sdf_grad_stride(desc),
        d_sdf_hat, loss, s);
    if (e != cudaSuccess || desc->feat_layout != PSDF_FEAT_TRIPLANE) return cuda_status(e);
    const size_t off = bf16_feat_offset(desc);
    e = psdf::launch_plane_reg(
        reinterpret_cast<const float4*>(static_cast<const uint8_t*>(packed_values) + off),
        tri_texels(desc), lam_features,
        reinterpret_cast<float4*>(static_cast<uint8_t*>(grad_grid) + off), loss ? loss + 3 : nullptr,
        s);
    return cuda_status(e);
}

psdf_status psdf_probe_smoothness(const psdf_probe_desc* desc, const float* coeffs, float lam,
                                  float* grad, float* loss, void* stream)
{
    const psdf_status st = check_probe_desc(desc);
    if (st != PSDF_OK) return st;
    if (desc->dtype != PSDF_F32) return PSDF_ERR_BAD_DTYPE;
    const int per = desc->sh_l * desc->sh_l * desc->n_ang;
    if (per % 4 != 0) return PSDF_ERR_UNSUPPORTED;
    if (!coeffs || !grad || !(lam >= 0.0f)) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(coeffs) || !aligned16(grad) ||
        (loss && (reinterpret_cast<uintptr_t>(loss) & 3u)))
        return PSDF_ERR_MISALIGNED;
    return cuda_status(psdf::launch_probe_reg(reinterpret_cast<const float4*>(coeffs), desc->dims,
                                              per / 4, lam, reinterpret_cast<float4*>(grad),
                                              loss, static_cast<cudaStream_t>(stream)));
}

// ---------------------------------------------------------------------------
// Learned sample proposal
// ---------------------------------------------------------------------------

namespace {

psdf_status check_proposal_desc(const psdf_proposal_desc* d)
{
    if (!d) return PSDF_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (d->occ_res[a] < 2 || d->occ_res[a] > 64) return PSDF_ERR_BAD_SHAPE;
    if (d->n_sub < 1 || d->n_sub > 32) return PSDF_ERR_BAD_SHAPE;
    if (!psdf::proposal_bins_supported(d->n_bins) || d->width != psdf::proposal_width())
        return PSDF_ERR_UNSUPPORTED;
    if (!(d->mix >= 0.0f && d->mix < 1.0f) || !(d->theta >= 0.0f)) return PSDF_ERR_INVALID_ARG;
    return PSDF_OK;
}

psdf_status grid_view(const psdf_grid* grid, psdf::GridView& g)
{
    if (!grid || !grid->values) return PSDF_ERR_INVALID_ARG;
    const psdf_grid_desc& gd = grid->desc;
    std::memset(&g, 0, sizeof(g));
    set_grid_view(gd, grid->values, g);
    for (int a = 0; a < 3; ++a) {
        g.R[a] = gd.dims[a];
        g.bmin[a] = gd.box_min[a];
        g.bmax[a] = gd.box_max[a];
        const volatile float ext = gd.box_max[a] - gd.box_min[a];
        g.sc[a] = static_cast<float>(gd.dims[a] - 1) / ext;
    }
    return PSDF_OK;
}

}  // namespace

psdf_status psdf_proposal_param_count(const psdf_proposal_desc* desc, int64_t* count)
{
    const psdf_status st = check_proposal_desc(desc);
    if (st != PSDF_OK) return st;
    if (!count) return PSDF_ERR_INVALID_ARG;
    *count = psdf::proposal_param_count(desc->n_bins);
    return PSDF_OK;
}

psdf_status psdf_occupancy_words(const int32_t occ_res[3], int64_t* words)
{
    if (!occ_res || !words) return PSDF_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (occ_res[a] < 2 || occ_res[a] > 64) return PSDF_ERR_BAD_SHAPE;
    const int res[3] = {occ_res[0], occ_res[1], occ_res[2]};
    *words = psdf::occupancy_words(res);
    return PSDF_OK;
}

psdf_status psdf_occupancy_build(const psdf_grid* grid, const int32_t occ_res[3],
                                 float threshold, uint32_t* occ_bits, void* stream)
{
    psdf::GridView g;
    psdf_status st = grid_view(grid, g);
    if (st != PSDF_OK) return st;
    int64_t words = 0;
    st = psdf_occupancy_words(occ_res, &words);
    if (st != PSDF_OK) return st;
    if (!occ_bits) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(occ_bits)) return PSDF_ERR_MISALIGNED;
    const int res[3] = {occ_res[0], occ_res[1], occ_res[2]};
    return cuda_status(psdf::launch_occupancy(g, res, threshold, occ_bits,
                                              static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_weight_histogram(const psdf_grid* grid, const psdf_render_params* params,
                                  const float* rays_o, const float* rays_d, int64_t n_rays,
                                  int32_t n_bins, float* hist, void* stream)
{
    if (!params || n_rays < 0) return PSDF_ERR_INVALID_ARG;
    if (!(params->tau > 0.0f) || params->n_samples < 1 || params->n_samples > 4096)
        return PSDF_ERR_BAD_SHAPE;
    if (n_bins < 1 || n_bins > 32 || params->n_samples % n_bins) return PSDF_ERR_BAD_SHAPE;
    psdf::RenderArgs A;
    std::memset(&A, 0, sizeof(A));
    psdf_status st = grid_view(grid, A.grid);
    if (st != PSDF_OK) return st;
    if (n_rays > 0 && (!rays_o || !rays_d || !hist)) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(rays_o) || !aligned16(rays_d) || !aligned16(hist)) return PSDF_ERR_MISALIGNED;
    if (n_rays == 0) return PSDF_OK;
    A.tau = params->tau;
    A.n_samples = params->n_samples;
    A.rays_o = rays_o;
    A.rays_d = rays_d;
    A.n_rays = n_rays;
    return cuda_status(
        psdf::launch_histogram(A, n_bins, hist, static_cast<cudaStream_t>(stream)));
}

namespace {

psdf_status proposal_launch(const psdf_grid* grid, const psdf_proposal_desc* desc,
                            const float* params, const uint32_t* occ, const float* rays_o,
                            const float* rays_d, int64_t n_rays, psdf::ProposalLaunch& L)
{
    psdf_status st = check_proposal_desc(desc);
    if (st != PSDF_OK) return st;
    std::memset(&L, 0, sizeof(L));
    st = grid_view(grid, L.grid);
    if (st != PSDF_OK) return st;
    if (!params || !occ || n_rays < 0) return PSDF_ERR_INVALID_ARG;
    if (n_rays > 0 && (!rays_o || !rays_d)) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(params) || !aligned16(occ) || !aligned16(rays_o) || !aligned16(rays_d))
        return PSDF_ERR_MISALIGNED;
    for (int a = 0; a < 3; ++a) L.occ_res[a] = desc->occ_res[a];
    L.n_bins = desc->n_bins;
    L.n_sub = desc->n_sub;
    L.occ_bits = occ;
    L.params = params;
    L.mix = desc->mix;
    L.theta = desc->theta;
    L.rays_o = rays_o;
    L.rays_d = rays_d;
    L.n_rays = n_rays;
    return PSDF_OK;
}

}  // namespace

psdf_status psdf_proposal_forward(const psdf_grid* grid, const psdf_proposal_desc* desc,
                                  const float* params, const uint32_t* occ_bits,
                                  const float* rays_o,
                                  const float* rays_d, int64_t n_rays, int32_t n_out,
                                  float* t_samples, float* probs, void* stream)
{
    psdf::ProposalLaunch L;
    psdf_status st = proposal_launch(grid, desc, params, occ_bits, rays_o, rays_d, n_rays, L);
    if (st != PSDF_OK) return st;
    if (n_out < 1 || n_out > 4096) return PSDF_ERR_BAD_SHAPE;
    if (n_rays > 0 && !t_samples && !probs) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(t_samples) || !aligned16(probs)) return PSDF_ERR_MISALIGNED;
    if (n_rays == 0) return PSDF_OK;
    L.n_out = n_out;
    L.t_samples = t_samples;
    L.probs = probs;
    return cuda_status(psdf::launch_proposal_forward(L, static_cast<cudaStream_t>(stream)));
}

psdf_status psdf_proposal_backward(const psdf_grid* grid, const psdf_proposal_desc* desc,
                                   const float* params, const uint32_t* occ_bits,
                                   const float* rays_o,
                                   const float* rays_d, int64_t n_rays, const float* hist,
                                   float min_mass, float scale, float* grad_params, float* loss,
                                   void* stream)
{
    psdf::ProposalLaunch L;
    psdf_status st = proposal_launch(grid, desc, params, occ_bits, rays_o, rays_d, n_rays, L);
    if (st != PSDF_OK) return st;
    if (!grad_params || (n_rays > 0 && !hist)) return PSDF_ERR_INVALID_ARG;
    if (!aligned16(hist) || !aligned16(grad_params) || !aligned16(loss)) return PSDF_ERR_MISALIGNED;
    if (n_rays == 0) return PSDF_OK;
    L.hist = hist;
    L.min_mass = min_mass;
    L.scale = scale;
    L.grad = grad_params;
    L.loss = loss;
    return cuda_status(psdf::launch_proposal_backward(L, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
