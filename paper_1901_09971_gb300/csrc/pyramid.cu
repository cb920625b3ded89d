// Image pyramid with Sobel gradients for RLOF tracking (arXiv 1901.09971, Section 2,
// "Sparse point tracking": RLOF works coarse to fine over an image pyramid that the
// paper does not define).
//
// Definition used: level l+1 = 2x2 block means of level l (sizes floor(W_l/2) x
// floor(H_l/2)); Ix, Iy = Sobel / 8 with clamped borders. Level-l pixel (x, y) is
// therefore exactly (sum of the 2^l x 2^l block of level-0 bytes at (2^l x, 2^l y))
// / 4^l: an integer times a power of two, exact in FP32 for every level this
// library allows, and so are the Sobel sums. Hence every level can be computed
// straight from the uint8 frame, independently of the others, in one launch:
// each CTA owns one tile of one level, stages the level-0 bytes under the tile plus
// a one-pixel level-l halo in shared memory, forms the exact level values there,
// and writes I (and Ix, Iy) with coalesced rows. FP16 storage rounds each exact
// value once.
#include "common.cuh"
#include "batch.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kSmemBytes = 40 * 1024;

__host__ __device__ inline int tile_w(int l) { return 64 >> (l < 4 ? l : 4); }
__host__ __device__ inline int tile_h(int l) { return l == 0 ? 16 : (l == 1 ? 8 : 4); }

// CTAs of one frame's pyramid: coarsest level first (those CTAs do the most work).
__host__ __device__ inline int level_ctas(int W, int H, int l)
{
    const int w = W >> l, h = H >> l;
    return ((w + tile_w(l) - 1) / tile_w(l)) * ((h + tile_h(l) - 1) / tile_h(l));
}

__host__ __device__ inline int frame_ctas(int W, int H, int levels)
{
    int n = 0;
    for (int l = 0; l < levels; ++l) n += level_ctas(W, H, l);
    return n;
}

}  // namespace

namespace dgf {

// One launch builds every level of up to kMaxFrames pyramids; CTAs are assigned
// frame by frame (cta_begin is the prefix count).
template <typename TS>
__global__ void __launch_bounds__(kThreads) pyramid_kernel(const __grid_constant__ PyrBatch a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int f = 0;  // frame of this CTA (binary search over the prefix counts)
    for (int lo = 0, hi = a.n_frames - 1; lo <= hi;) {
        const int mid = (lo + hi) >> 1;
        if (a.frames[mid].cta_begin <= (int)blockIdx.x) {
            f = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    const PyrFrame& F = a.frames[f];
    int t = blockIdx.x - F.cta_begin, l = a.levels - 1;
    for (; l > 0; --l) {
        const int n = level_ctas(F.W, F.H, l);
        if (t < n) break;
        t -= n;
    }
    LevelGeom d;
    level_geom(F.W, F.H, a.levels, (int)sizeof(TS), l, &d);
    const int tw = tile_w(l), th = tile_h(l);
    const int tiles_x = (d.W + tw - 1) / tw;
    const int tx0 = (t % tiles_x) * tw, ty0 = (t / tiles_x) * th;
    const int s = 1 << l;
    const int vw = tw + 2, vh = th + 2;  // level values incl. the halo
    const int rw = vw * s, rh = vh * s;  // level-0 bytes under them
    float* val = reinterpret_cast<float*>(smem);
    unsigned char* raw = smem + ((vw * vh * 4 + 15) & ~15);
    const int gx0 = (tx0 - 1) * s, gy0 = (ty0 - 1) * s;

    // 1. stage the level-0 bytes (only those inside the frame are ever used)
    for (int i = threadIdx.x; i < rw * rh; i += blockDim.x) {
        const int ry = i / rw, rx = i - ry * rw;
        const int gx = gx0 + rx, gy = gy0 + ry;
        raw[i] = (gx >= 0 && gx < F.W && gy >= 0 && gy < F.H) ? F.img[(size_t)gy * F.pitch + gx] : 0;
    }
    __syncthreads();
    // 2. exact level-l values on the tile and its halo (inside the level only)
    const float scale = 1.0f / (float)(s * s);  // 4^-l, exact
    for (int i = threadIdx.x; i < vw * vh; i += blockDim.x) {
        const int vy = i / vw, vx = i - vy * vw;
        const int x = tx0 - 1 + vx, y = ty0 - 1 + vy;
        float v = 0.f;
        if (x >= 0 && x < d.W && y >= 0 && y < d.H) {
            int sum = 0;
            const unsigned char* b = raw + (vy * s) * rw + vx * s;
            for (int yy = 0; yy < s; ++yy)
                for (int xx = 0; xx < s; ++xx) sum += b[yy * rw + xx];
            v = (float)sum * scale;
        }
        val[i] = v;
    }
    __syncthreads();
    // 3. write the tile: I, and Sobel / 8 with clamped neighbours
    TS* I = reinterpret_cast<TS*>(F.base + d.off_I);
    TS* Ix = reinterpret_cast<TS*>(F.base + d.off_Ix);
    TS* Iy = reinterpret_cast<TS*>(F.base + d.off_Iy);
    for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
        const int ty = i / tw, tx = i - ty * tw;
        const int x = tx0 + tx, y = ty0 + ty;
        if (x >= d.W || y >= d.H) continue;
        const size_t o = (size_t)y * d.pitch + x;
        st(I + o, val[(ty + 1) * vw + tx + 1]);
        if (F.with_grad) {
            // region index of a clamped level coordinate
            const int xm = max(x - 1, 0) - (tx0 - 1), xp = min(x + 1, d.W - 1) - (tx0 - 1);
            const int ym = max(y - 1, 0) - (ty0 - 1), yp = min(y + 1, d.H - 1) - (ty0 - 1);
            const int xc = tx + 1, yc = ty + 1;
            const float gx = (val[ym * vw + xp] - val[ym * vw + xm]) + 2.f * (val[yc * vw + xp] - val[yc * vw + xm]) +
                             (val[yp * vw + xp] - val[yp * vw + xm]);
            const float gy = (val[yp * vw + xm] - val[ym * vw + xm]) + 2.f * (val[yp * vw + xc] - val[ym * vw + xc]) +
                             (val[yp * vw + xp] - val[ym * vw + xp]);
            st(Ix + o, gx * 0.125f);
            st(Iy + o, gy * 0.125f);
        }
    }
}

// Shared memory of the most demanding level (the coarsest).
size_t pyramid_smem(int levels)
{
    size_t smem = 0;
    for (int l = 0; l < levels; ++l) {
        const size_t vw = tile_w(l) + 2, vh = tile_h(l) + 2, s = (size_t)1 << l;
        const size_t need = round_up(vw * vh * 4, 16) + vw * vh * s * s;
        smem = smem > need ? smem : need;
    }
    return smem;
}

// Fills the CTA prefix counts and launches one pyramid build for every frame.
int launch_pyramids(PyrBatch& a, int storage, cudaStream_t stream)
{
    int ctas = 0;
    for (int f = 0; f < a.n_frames; ++f) {
        a.frames[f].cta_begin = ctas;
        ctas += frame_ctas(a.frames[f].W, a.frames[f].H, a.levels);
    }
    const size_t smem = pyramid_smem(a.levels);
    if (smem > (size_t)kSmemBytes) return DGF_ERR_ARG;
    if (ctas == 0) return DGF_OK;
    if (storage == DGF_F32)
        pyramid_kernel<float><<<ctas, kThreads, smem, stream>>>(a);
    else
        pyramid_kernel<__half><<<ctas, kThreads, smem, stream>>>(a);
    return launch_status();
}

}  // namespace dgf

extern "C" int dgf_pyramid_layout_get(int W, int H, int levels, int storage, int with_grad,
                                      dgf_pyramid_layout* out)
{
    if (!out || W < 1 || H < 1 || levels < 1 || levels > DGF_MAX_LEVELS ||
        (storage != DGF_F32 && storage != DGF_F16))
        return DGF_ERR_ARG;
    dgf_pyramid_layout L = {};
    L.levels = levels;
    L.storage = storage;
    L.with_grad = with_grad ? 1 : 0;
    const int es = storage == DGF_F32 ? 4 : 2;
    for (int l = 0; l < levels; ++l) {
        dgf::LevelGeom g;
        if (!dgf::level_geom(W, H, levels, es, l, &g)) return DGF_ERR_ARG;
        L.W[l] = g.W;
        L.H[l] = g.H;
        L.pitch[l] = g.pitch;
        L.off_I[l] = g.off_I;
        L.off_Ix[l] = L.with_grad ? g.off_Ix : 0;
        L.off_Iy[l] = L.with_grad ? g.off_Iy : 0;
        L.bytes = L.with_grad ? g.bytes_all : g.bytes_intensity;
    }
    *out = L;
    return DGF_OK;
}

extern "C" size_t dgf_pyramid_bytes(int W, int H, int levels, int storage, int with_grad)
{
    dgf_pyramid_layout L;
    return dgf_pyramid_layout_get(W, H, levels, storage, with_grad, &L) == DGF_OK ? L.bytes : 0;
}

extern "C" int pyramid_build(const uint8_t* img, int W, int H, int pitch, int levels, int storage,
                             int with_grad, void* pyr, size_t pyr_bytes, cudaStream_t stream)
{
    dgf_pyramid_layout L;
    if (!img || !pyr || pitch < W) return DGF_ERR_ARG;
    int rc = dgf_pyramid_layout_get(W, H, levels, storage, with_grad, &L);
    if (rc != DGF_OK) return rc;
    if (!dgf::aligned(pyr, 256)) return DGF_ERR_ARG;
    if (pyr_bytes < L.bytes) return DGF_ERR_WORKSPACE;
    dgf::PyrBatch a = {};
    a.levels = levels;
    a.n_frames = 1;
    a.frames[0] = dgf::PyrFrame{img, W, H, pitch, L.with_grad, static_cast<char*>(pyr), 0};
    return dgf::launch_pyramids(a, storage, stream);
}
