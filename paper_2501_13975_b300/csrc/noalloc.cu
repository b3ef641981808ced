// gs2_render_noalloc: projection, tile binning/sort and compositing of one
// view without allocating device memory.
//
// Some callers cannot call cudaMalloc: a plugin or callback run by a host
// application that owns all device memory and does not let its plugins
// allocate, or a real-time loop that must not pay allocation latency or risk
// an out-of-memory failure halfway through a run.  This entry point needs no
// gs2_ctx: its sorting scratch lives in one fixed-size array compiled into the
// library (GS2_NOALLOC_SCRATCH_BYTES, about 9 MB), which every GPU that loads
// the library holds until the process exits.  The caller still passes the
// projection buffer, the image and the raster state.
//
// Set-up: the first call on a device looks up the device address of the
// array (cudaGetSymbolAddress) with that device current; make that first call
// before any stream capture.  All calls share the one array, so calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race and must be serialised by the caller.
#include <mutex>

#include "common.cuh"

#define NA_SORT_BLOCKS (148 * 4)

// carve-up of the scratch array (byte offsets, each 256-aligned)
#define NA_KEYS_BYTES (4ull * GS2_NOALLOC_MAX_PAIRS)
#define NA_VALS_BYTES (4ull * GS2_NOALLOC_MAX_PAIRS)
#define NA_GHIST_BYTES (4ull * (256 * NA_SORT_BLOCKS + 256))
#define NA_SS_BYTES (8ull * 1024)   // the tiles-touched scan's state (GS2_SS_WORDS words)
#define NA_RANGES_BYTES (8ull * GS2_NOALLOC_MAX_TILES)
#define NA_OFF_KEYS0 0ull
#define NA_OFF_KEYS1 (NA_OFF_KEYS0 + NA_KEYS_BYTES)
#define NA_OFF_VALS0 (NA_OFF_KEYS1 + NA_KEYS_BYTES)
#define NA_OFF_VALS1 (NA_OFF_VALS0 + NA_VALS_BYTES)
#define NA_OFF_GHIST (NA_OFF_VALS1 + NA_VALS_BYTES)
#define NA_OFF_SS (NA_OFF_GHIST + NA_GHIST_BYTES)
#define NA_OFF_RANGES (NA_OFF_SS + NA_SS_BYTES)
#define NA_OFF_COUNT (NA_OFF_RANGES + NA_RANGES_BYTES)
#define NA_OFF_STATUS (NA_OFF_COUNT + 256ull)
#define NA_TOTAL (NA_OFF_STATUS + 256ull)

static_assert(NA_TOTAL == GS2_NOALLOC_SCRATCH_BYTES, "scratch size in gs2.h must match the carve-up");
static_assert(4ull * GS2_SS_WORDS <= NA_SS_BYTES, "scan state fits its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[GS2_NOALLOC_SCRATCH_BYTES];

#define NA_MAX_DEVICES 64
static unsigned char *g_scratch_addr[NA_MAX_DEVICES];
static std::mutex g_scratch_mu;

// device address of the scratch array on the current device (looked up once per device)
static cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

extern "C" gs2_status gs2_render_noalloc(const gs2_config *cfg, const gs2_scene *scene, const gs2_camera *cam,
                                         void *proj, float *image, void *raster_state, uint32_t *status_out,
                                         gs2_stream stream) {
    if (!scene || !cam || !proj || !image || !raster_state) return GS2_ERR_ARG;
    if (scene->n < 0 || scene->sh_degree < 0) return GS2_ERR_ARG;
    if (scene->sh_degree > 3) return GS2_ERR_UNSUPPORTED;
    if (scene->n > 0 && !(scene->mean && scene->quat && scene->scale && scene->opacity && scene->sh))
        return GS2_ERR_ARG;
    if (cam->width < 1 || cam->height < 1 || !(cam->fx > 0.f) || !(cam->fy > 0.f)) return GS2_ERR_ARG;
    const int tiles_x = (cam->width + GS2_TILE - 1) / GS2_TILE, tiles_y = (cam->height + GS2_TILE - 1) / GS2_TILE;
    if ((long long)tiles_x * tiles_y > GS2_NOALLOC_MAX_TILES) return GS2_ERR_SHAPE;
    gs2_config c;
    if (cfg) {
        std::string err;   // the same checks as gs2_create / gs2_set_config, before any device call
        if (!cfg_ok(cfg, err)) return GS2_ERR_ARG;
        c = *cfg;
    } else {
        gs2_config_default(&c);
    }
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return GS2_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;

    // a context view onto the fixed array: nothing here allocates
    gs2_ctx v{};
    v.cfg = c;
    v.max_pairs = GS2_NOALLOC_MAX_PAIRS;
    v.nb_sort = NA_SORT_BLOCKS;
    v.sort_rows = 4;
    v.keys[0] = (uint32_t *)(base + NA_OFF_KEYS0);
    v.keys[1] = (uint32_t *)(base + NA_OFF_KEYS1);
    v.vals[0] = (uint32_t *)(base + NA_OFF_VALS0);
    v.vals[1] = (uint32_t *)(base + NA_OFF_VALS1);
    v.ghist = (uint32_t *)(base + NA_OFF_GHIST);
    v.sort_state = (uint32_t *)(base + NA_OFF_SS);
    v.ranges = (uint2 *)(base + NA_OFF_RANGES);
    v.d_count = (uint32_t *)(base + NA_OFF_COUNT);
    v.d_status = (uint32_t *)(base + NA_OFF_STATUS);
    v.tiles_x = tiles_x;
    v.tiles_y = tiles_y;

    // the status word accumulates bits: it must start at zero for this call
    if (cudaMemsetAsync(v.d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return GS2_ERR_CUDA;
    const DevScene sc = make_devscene(scene);
    const DevCam dc = make_devcam(cam);
    ProjView pv = proj_view(proj, scene->n);
    if (launch_project(sc, dc, c, pv, tiles_x, tiles_y, st, v.d_status) != cudaSuccess) return GS2_ERR_CUDA;
    if (launch_bin_sort(&v, pv, scene->n, tiles_x, tiles_y, st, nullptr) != cudaSuccess) return GS2_ERR_CUDA;
    if (launch_raster(&v, pv, dc, c, image, raster_view(raster_state, cam->width, cam->height), st) != cudaSuccess)
        return GS2_ERR_CUDA;
    if (status_out &&
        cudaMemcpyAsync(status_out, v.d_status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return GS2_ERR_CUDA;
    return GS2_OK;
}
