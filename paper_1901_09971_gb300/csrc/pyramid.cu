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

namespace {

struct LevelDesc {
    int W, H, pitch;  // level size and row pitch (elements)
    int tw, th;       // tile size (level pixels)
    int tiles_x;      // tiles per row
    int cta_begin;    // first CTA of this level in the flattened grid
    size_t off_I, off_Ix, off_Iy;
};

struct PyrArgs {
    const uint8_t* img;
    int W, H, pitch, levels, with_grad;
    char* base;
    LevelDesc lv[DGF_MAX_LEVELS];
    int cta_end;
};

constexpr int kThreads = 256;
constexpr int kSmemBytes = 40 * 1024;

int tile_w(int l) { return 64 >> (l < 4 ? l : 4); }
int tile_h(int l) { return l == 0 ? 16 : (l == 1 ? 8 : 4); }

template <typename TS>
__global__ void __launch_bounds__(kThreads) pyramid_kernel(PyrArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // CTAs are ordered coarsest level first (they do the most work per CTA)
    int l = a.levels - 1;
    for (int k = 0; k < a.levels; ++k)
        if ((int)blockIdx.x >= a.lv[k].cta_begin) { l = k; break; }
    const LevelDesc& d = a.lv[l];
    const int t = blockIdx.x - d.cta_begin;
    const int tx0 = (t % d.tiles_x) * d.tw, ty0 = (t / d.tiles_x) * d.th;
    const int s = 1 << l;
    const int vw = d.tw + 2, vh = d.th + 2;  // level values incl. the halo
    const int rw = vw * s, rh = vh * s;      // level-0 bytes under them
    float* val = reinterpret_cast<float*>(smem);
    unsigned char* raw = smem + ((vw * vh * 4 + 15) & ~15);
    const int gx0 = (tx0 - 1) * s, gy0 = (ty0 - 1) * s;

    // 1. stage the level-0 bytes (only those inside the frame are ever used)
    for (int i = threadIdx.x; i < rw * rh; i += blockDim.x) {
        const int ry = i / rw, rx = i - ry * rw;
        const int gx = gx0 + rx, gy = gy0 + ry;
        raw[i] = (gx >= 0 && gx < a.W && gy >= 0 && gy < a.H) ? a.img[(size_t)gy * a.pitch + gx] : 0;
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
    TS* I = reinterpret_cast<TS*>(a.base + d.off_I);
    TS* Ix = reinterpret_cast<TS*>(a.base + d.off_Ix);
    TS* Iy = reinterpret_cast<TS*>(a.base + d.off_Iy);
    for (int i = threadIdx.x; i < d.tw * d.th; i += blockDim.x) {
        const int ty = i / d.tw, tx = i - ty * d.tw;
        const int x = tx0 + tx, y = ty0 + ty;
        if (x >= d.W || y >= d.H) continue;
        const size_t o = (size_t)y * d.pitch + x;
        dgf::st(I + o, val[(ty + 1) * vw + tx + 1]);
        if (a.with_grad) {
            // region index of a clamped level coordinate
            const int xm = max(x - 1, 0) - (tx0 - 1), xp = min(x + 1, d.W - 1) - (tx0 - 1);
            const int ym = max(y - 1, 0) - (ty0 - 1), yp = min(y + 1, d.H - 1) - (ty0 - 1);
            const int xc = tx + 1, yc = ty + 1;
            const float gx = (val[ym * vw + xp] - val[ym * vw + xm]) + 2.f * (val[yc * vw + xp] - val[yc * vw + xm]) +
                             (val[yp * vw + xp] - val[yp * vw + xm]);
            const float gy = (val[yp * vw + xm] - val[ym * vw + xm]) + 2.f * (val[yp * vw + xc] - val[ym * vw + xc]) +
                             (val[yp * vw + xp] - val[ym * vw + xp]);
            dgf::st(Ix + o, gx * 0.125f);
            dgf::st(Iy + o, gy * 0.125f);
        }
    }
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

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
    const size_t es = storage == DGF_F32 ? 4 : 2;
    size_t plane[DGF_MAX_LEVELS];
    int w = W, h = H;
    for (int l = 0; l < levels; ++l) {
        if (w < 1 || h < 1) return DGF_ERR_ARG;
        L.W[l] = w;
        L.H[l] = h;
        L.pitch[l] = (int)round_up((size_t)w, 128 / es);
        plane[l] = round_up((size_t)L.pitch[l] * h * es, 256);
        w /= 2;
        h /= 2;
    }
    size_t off = 0;
    for (int l = 0; l < levels; ++l) { L.off_I[l] = off; off += plane[l]; }
    if (L.with_grad) {
        for (int l = 0; l < levels; ++l) { L.off_Ix[l] = off; off += plane[l]; }
        for (int l = 0; l < levels; ++l) { L.off_Iy[l] = off; off += plane[l]; }
    }
    L.bytes = off;
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
    PyrArgs a = {};
    a.img = img;
    a.W = W;
    a.H = H;
    a.pitch = pitch;
    a.levels = levels;
    a.with_grad = L.with_grad;
    a.base = static_cast<char*>(pyr);
    int ctas = 0;
    for (int l = levels - 1; l >= 0; --l) {
        LevelDesc& d = a.lv[l];
        d.W = L.W[l];
        d.H = L.H[l];
        d.pitch = L.pitch[l];
        d.tw = tile_w(l);
        d.th = tile_h(l);
        d.tiles_x = (d.W + d.tw - 1) / d.tw;
        d.cta_begin = ctas;
        d.off_I = L.off_I[l];
        d.off_Ix = L.off_Ix[l];
        d.off_Iy = L.off_Iy[l];
        ctas += d.tiles_x * ((d.H + d.th - 1) / d.th);
    }
    a.cta_end = ctas;
    // shared memory of the most demanding level (the coarsest)
    size_t smem = 0;
    for (int l = 0; l < levels; ++l) {
        const size_t vw = tile_w(l) + 2, vh = tile_h(l) + 2, s = (size_t)1 << l;
        smem = smem > round_up(vw * vh * 4, 16) + vw * vh * s * s ? smem : round_up(vw * vh * 4, 16) + vw * vh * s * s;
    }
    if (smem > (size_t)kSmemBytes) return DGF_ERR_ARG;
    if (storage == DGF_F32)
        pyramid_kernel<float><<<ctas, kThreads, smem, stream>>>(a);
    else
        pyramid_kernel<__half><<<ctas, kThreads, smem, stream>>>(a);
    return dgf::launch_status();
}
