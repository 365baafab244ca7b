// cgs_render_forward_static: the forward render of one small view with its scratch memory in
// a fixed, file-scope device array instead of a caller-allocated workspace.
//
// For callers that cannot allocate device memory: a host application that owns all device
// memory and forbids allocation inside its frame loop, a plugin that is handed only its input
// and output buffers, or a process without a tensor library to size and hold a workspace.
// They pass inputs and outputs; the intermediate state (sorted lists, records, counters)
// lives in g_static_ws, which every GPU that loads this library keeps until the process exits.
#include "common.cuh"

namespace cgs {

// The scratch of the static variant.  In host code this name is only a stand-in for the
// device symbol: the device address comes from cudaGetSymbolAddress (static_base).
static __device__ __align__(256) unsigned char g_static_ws[CGS_STATIC_WORKSPACE_BYTES];

// Device address of g_static_ws on the current device, looked up with that device current on
// every call (nothing is cached, so the address stays right after a device reset reloads the
// module).  The first lookup on a device loads the library's module there, which is why the
// first call on a device should come before any stream capture.  Returns nullptr if the
// lookup fails.
static void* static_base()
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess) return nullptr;
    return p;
}

// Writes the frame's status as a CGS_* code into *out (device memory).
__global__ void k_static_status(const Header* hdr, int32_t* out)
{
    const uint32_t s = hdr->status;
    *out = (s & ST_SPIN) ? CGS_ERR_SPIN_TIMEOUT
                         : ((s & ST_CAPACITY) ? CGS_ERR_CAPACITY : ((s & ST_UNSUPPORTED) ? CGS_ERR_UNSUPPORTED : CGS_OK));
}

}  // namespace cgs

using namespace cgs;

extern "C" int32_t cgs_render_forward_static(const cgs_scene* scene, const cgs_config* cfg, const cgs_camera* d_cam,
                                             int32_t width, int32_t height, const int32_t* d_view_block,
                                             const int8_t* d_levels, float* d_image, float* d_final_T,
                                             uint32_t* d_n_contrib, int32_t* d_status, void* stream)
{
    if (!scene || !cfg || width < 1 || height < 1) return CGS_ERR_INVALID_ARGUMENT;
    if ((int64_t)width * height > CGS_STATIC_MAX_PIXELS || scene->n > CGS_STATIC_MAX_GAUSSIANS ||
        scene->n_blocks > CGS_STATIC_MAX_BLOCKS)
        return CGS_ERR_TOO_LARGE;
    cgs_frame f;
    f.ws = nullptr;
    f.ws_bytes = CGS_STATIC_WORKSPACE_BYTES;
    f.n_views = 1;
    f.width = width;
    f.height = height;
    f.tile = cfg->tile;
    f.n_blocks = scene->n_blocks;
    f.flags = 0;
    f.n_cap = scene->n > 0 ? scene->n : 1;
    f.k_cap = CGS_STATIC_MAX_ENTRIES;
    const int64_t need = cgs_frame_workspace_bytes(1, width, height, cfg->tile, scene->n_blocks, f.n_cap, f.k_cap);
    if (need <= 0) return CGS_ERR_INVALID_ARGUMENT;
    if (need > CGS_STATIC_WORKSPACE_BYTES) return CGS_ERR_TOO_LARGE;
    void* base = static_base();
    if (!base) return CGS_ERR_CUDA;
    f.ws = base;
    const int32_t rc = cgs_render_forward(scene, &f, cfg, d_cam, d_view_block, d_levels, d_image, d_final_T,
                                          d_n_contrib, stream);
    if (rc != CGS_OK) return rc;
    if (d_status) {
        k_static_status<<<1, 1, 0, (cudaStream_t)stream>>>(reinterpret_cast<const Header*>(base), d_status);
        if (cudaGetLastError() != cudaSuccess) return CGS_ERR_CUDA;
    }
    return CGS_OK;
}
