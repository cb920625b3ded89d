// Image pyramid with Sobel gradients for RLOF tracking (arXiv 1901.09971, Section 2,
// "Sparse point tracking": RLOF works coarse to fine over an image pyramid that the
// paper does not define).
//
// Definition used: level l+1 = 2x2 block means of level l (sizes floor(W_l/2) x
// floor(H_l/2)); Ix, Iy = Sobel / 8 with clamped borders. Every level value is an
// integer byte sum times 4^-l and every Sobel sum a small multiple of it, so all of
// them are exact in FP32 (FP16 storage rounds each exact value once).
//
// One CTA owns a tile of level 0 (128 x 64 pixels for up to 4 levels, 64 x 32 beyond)
// and produces the matching tile of every level. It stages the frame bytes under
// the tile plus a halo of 2^(L-1) pixels (enough for a one-pixel halo at the
// coarsest level) in shared memory: one bulk asynchronous copy per row when the
// frame's base, pitch and width are multiples of 16 bytes, otherwise asynchronous
// 4-byte copies (cp.async) of the aligned words that hold them (frame rows need not
// start on any boundary, so each staged row keeps its own misalignment, 0..3 bytes,
// and every read adds it). Then the CTA walks down the levels, forming each level's
// values on its halo'd region from the previous one with 2x2 means. Outputs are
// written by vertical strips: a group of threads owns a band of rows and a thread a
// few columns (four at level 0), sliding down the band with the rows above and below
// in registers, so every staged row is read once per thread and a warp's loads are
// consecutive words; each row's I, Ix, Iy are written with coalesced stores (16 bytes
// a thread at level 0). Columns and rows outside the level are clamped to it (the
// Sobel stencil's border rule) by precomputed column offsets and a clamped row index,
// one code path for every tile. Tiles on the frame's edge also write the planes'
// replicated borders (kApron pixels wide; the clamped values, so that tracking reads
// its taps without clamping). The frame is read about once from DRAM and every
// output byte is written once.
#include "common.cuh"
#include "batch.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Level-0 tile: 128 x 64 pixels up to 4 levels (a warp's 32 lanes x 4 columns a row);
// 64 x 32 beyond, where the halo grows to 16 or 32 pixels and a single frame needs
// the smaller tiles to spread over the SMs (one 1242x375 frame: 240 blocks).
__host__ __device__ constexpr int tile_w(int levels) { return levels <= 4 ? 128 : 64; }
__host__ __device__ constexpr int tile_h(int levels) { return levels <= 4 ? 64 : 32; }
__host__ __device__ constexpr int halo(int levels) { return levels >= 2 ? 1 << (levels - 1) : 1; }
__host__ __device__ constexpr int region_w(int levels) { return tile_w(levels) + 2 * halo(levels); }
__host__ __device__ constexpr int region_h(int levels) { return tile_h(levels) + 2 * halo(levels); }
// staged row pitch: the region's bytes plus up to 15 bytes of row offset on either
// side (bulk copies move 16-byte-aligned spans), a multiple of 16
__host__ __device__ constexpr int region_pitch(int levels) { return (region_w(levels) + 32 + 15) & ~15; }

__host__ __device__ inline int frame_ctas(int W, int H, int levels)
{
    return ((W + tile_w(levels) - 1) / tile_w(levels)) * ((H + tile_h(levels) - 1) / tile_h(levels));
}

__host__ __device__ constexpr size_t round16(size_t v) { return (v + 15) & ~(size_t)15; }

// Shared memory of one CTA: the staged byte rows, then the float regions of levels 1..L-1.
inline size_t smem_bytes(int levels)
{
    const int RW = region_w(levels), RH = region_h(levels);
    size_t off = round16((size_t)region_pitch(levels) * RH);
    for (int l = 1; l < levels; ++l) off += round16((size_t)(RW >> l) * (RH >> l) * 4);
    return off;
}

template <typename TS>
__device__ __forceinline__ void store4(TS* p, float a, float b, float c, float d);
template <>
__device__ __forceinline__ void store4<float>(float* p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void store4<__half>(__half* p, float a, float b, float c, float d)
{
    __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
    uint2 v;
    v.x = *reinterpret_cast<unsigned*>(&lo);
    v.y = *reinterpret_cast<unsigned*>(&hi);
    *reinterpret_cast<uint2*>(p) = v;
}

template <typename TS>
__device__ __forceinline__ void store2(TS* p, float a, float b);
template <>
__device__ __forceinline__ void store2<float>(float* p, float a, float b)
{
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void store2<__half>(__half* p, float a, float b)
{
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
}

// Staged region rows: byte (r, c) of the halo'd region (frame pixel (gx0 + c,
// gy0 + r)) sits at raw[r * RWP + mis(r) + c]. BULK (bulk row copies): every row has
// the same offset, gx0 mod 16, which is (-h) mod 16 since tiles start on multiples of
// 64 columns. Word copies: mis(r) is the misalignment of that frame row's byte gx0
// (rows advance by the pitch, so it steps by pitch mod 4, mask 3).
template <int L, bool BULK>
struct Staged {
    static constexpr int RWP = region_pitch(L);
    const unsigned char* raw;
    unsigned mis0, pmod;  // word copies only
    __device__ __forceinline__ const unsigned char* row(int r) const
    {
        if constexpr (BULK) {
            constexpr unsigned kBulkMis = (unsigned)(-halo(L)) & 15u;
            return raw + r * RWP + kBulkMis;
        } else {
            return raw + r * RWP + ((mis0 + (unsigned)r * pmod) & 3u);
        }
    }
};

}  // namespace

namespace dgf {

constexpr int kRun = 4;                 // border values a thread writes
constexpr int kRuns = kApron / kRun;    // threads a border row or column
static_assert(kApron % kRun == 0, "border rows of whole runs");

// kRun copies of v at p[0], p[step], ..., p[(kRun - 1) step].
template <typename TS>
__device__ __forceinline__ void fill_strided(TS* p, ptrdiff_t step, float v)
{
#pragma unroll
    for (int k = 0; k < kRun; ++k) st(p + k * step, v);
}
// kRun copies of v at p[0 .. kRun), p 16-byte aligned (FP32) or 8-byte aligned
// (FP16): one vector store.
__device__ __forceinline__ void fill_run(float* p, float v) { *reinterpret_cast<float4*>(p) = make_float4(v, v, v, v); }
__device__ __forceinline__ void fill_run(__half* p, float v)
{
    const __half2 h = __float2half2_rn(v);
    uint2 w;
    w.x = w.y = *reinterpret_cast<const unsigned*>(&h);
    *reinterpret_cast<uint2*>(p) = w;
}

// The replicated border (kApron pixels wide) that a tile on a level's edge owns:
// outside the level, beside the tile's columns [x0, xe] and rows [y0, ye] (its part
// of the level), every position takes the values at its clamped position, which
// lies in the tile. The left and right strips include the corner blocks. A border
// row of a side strip, or a border column of the top or bottom strip, repeats one
// value: kRuns threads share it, each forming the value from the data the block
// already holds (value(x, y, I, Ix, Iy) at tile pixel (x, y)) and writing kRun
// copies. Rows start 128-byte aligned at pixel 0, so the runs of a left border row
// (from pixel -kApron) are vector stores; neighbouring threads write neighbouring
// runs of a row, or the same run of neighbouring columns.
template <typename TS, typename Value>
__device__ __forceinline__ void apron_strips(TS* I, TS* Ix, TS* Iy, bool grad, int pitch, int W, int H, int x0,
                                             int y0, int xe, int ye, Value value)
{
    if (xe < x0 || ye < y0) return;  // the tile holds no pixel of this level
    const bool L = x0 == 0, R = xe == W - 1, T = y0 == 0, B = ye == H - 1;
    if (!(L || R || T || B)) return;
    const int ry0 = T ? -kApron : y0, ry1 = B ? H - 1 + kApron : ye;  // rows of the side strips
    const int sh = ry1 - ry0 + 1, tw = xe - x0 + 1;
    const int nL = L ? kRuns * sh : 0, nR = R ? kRuns * sh : 0, nT = T ? kRuns * tw : 0, nB = B ? kRuns * tw : 0;
    for (int i = threadIdx.x; i < nL + nR + nT + nB; i += blockDim.x) {
        float vI, vx, vy;
        if (i < nL + nR) {  // a run of a row of the left or right strip
            const bool left = i < nL;
            const int j = left ? i : i - nL;
            const int ay = ry0 + j / kRuns, run = j % kRuns;
            value(left ? 0 : W - 1, min(max(ay, 0), H - 1), vI, vx, vy);
            const ptrdiff_t o = (ptrdiff_t)ay * pitch + (left ? -kApron : W) + kRun * run;
            if (left) {
                fill_run(I + o, vI);
                if (grad) {
                    fill_run(Ix + o, vx);
                    fill_run(Iy + o, vy);
                }
            } else {
                fill_strided(I + o, 1, vI);
                if (grad) {
                    fill_strided(Ix + o, 1, vx);
                    fill_strided(Iy + o, 1, vy);
                }
            }
        } else {  // a run of a column of the top or bottom strip
            const int j = i - nL - nR;
            const bool top = j < nT;
            const int k = top ? j : j - nT;
            const int ax = x0 + k % tw, run = k / tw;
            value(ax, top ? 0 : H - 1, vI, vx, vy);
            const ptrdiff_t o = (ptrdiff_t)((top ? -kApron : H) + kRun * run) * pitch + ax;
            fill_strided(I + o, pitch, vI);
            if (grad) {
                fill_strided(Ix + o, pitch, vx);
                fill_strided(Iy + o, pitch, vy);
            }
        }
    }
}

// Level 0 of the tile: I and Sobel / 8 straight from the staged bytes. TX/4 threads
// share a row: thread t owns columns x .. x+3 (x = X0 + 4 (t mod TX/4)) of the band
// of TY / (256 / (TX/4)) rows numbered t / (TX/4) (a warp's band at TX = 128).
// For each of its columns and each row the lane forms the horizontal difference
// d = p(k+2) - p(k) and smoothing s = p(k) + 2 p(k+1) + p(k+2); sliding down the band
// it keeps those of the row above and of the current row, and with the row below's,
// Sobel x = d_above + 2 d + d_below and Sobel y = s_below - s_above (exact integers).
// INTERIOR: the halo'd region lies inside the frame, so no index needs clamping.
template <typename TS, bool INTERIOR, int TX, int TY, typename ST>
__device__ __forceinline__ void level0(const PyrFrame& F, const LevelGeom& g, const ST& R, int X0, int Y0, int h)
{
    TS* I = reinterpret_cast<TS*>(F.base + g.off_I);
    TS* Ix = reinterpret_cast<TS*>(F.base + g.off_Ix);
    TS* Iy = reinterpret_cast<TS*>(F.base + g.off_Iy);
    const int gx0 = X0 - h, gy0 = Y0 - h;
    constexpr int LPR = TX / 4, NB = kThreads / LPR;  // threads a row, bands
    constexpr int RPW = TY / NB;                       // rows a band
    static_assert(LPR <= 32 && TY % NB == 0, "a band of whole rows per thread group");
    const int lane = threadIdx.x % LPR, warp = threadIdx.x / LPR;
    const int x = X0 + 4 * lane;
    int col[6];  // staged columns of pixels x-1 .. x+4, clamped to the frame
#pragma unroll
    for (int j = 0; j < 6; ++j) col[j] = (INTERIOR ? x - 1 + j : min(max(x - 1 + j, 0), F.W - 1)) - gx0;
    auto load_row = [&](int y, int (&v)[6]) {
        const unsigned char* r = R.row((INTERIOR ? y : min(max(y, 0), F.H - 1)) - gy0);
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = r[col[j]];
    };
    const int y0 = Y0 + warp * RPW;
    int d0[4], s0[4], d1[4], s1[4], c1[4];  // row above and current row (c1: its pixels)
    {
        int p[6], q[6];
        load_row(y0 - 1, p);
        load_row(y0, q);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            d0[k] = p[k + 2] - p[k];
            s0[k] = p[k] + 2 * p[k + 1] + p[k + 2];
            d1[k] = q[k + 2] - q[k];
            s1[k] = q[k] + 2 * q[k + 1] + q[k + 2];
            c1[k] = q[k + 1];
        }
    }
    const bool full = INTERIOR || x + 3 < F.W;  // all four columns inside the frame
#pragma unroll 1
    for (int i = 0; i < RPW; ++i) {
        const int y = y0 + i;
        int q[6];
        load_row(y + 1, q);
        int d2[4], s2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            d2[k] = q[k + 2] - q[k];
            s2[k] = q[k] + 2 * q[k + 1] + q[k + 2];
        }
        if (INTERIOR || (y < F.H && x < F.W)) {
            float vI[4], vx[4], vy[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                vI[k] = (float)c1[k];
                vx[k] = (float)(d0[k] + 2 * d1[k] + d2[k]) * 0.125f;
                vy[k] = (float)(s2[k] - s0[k]) * 0.125f;
            }
            const size_t o = (size_t)y * g.pitch + x;
            if (full) {
                store4<TS>(I + o, vI[0], vI[1], vI[2], vI[3]);
                if (F.with_grad) {
                    store4<TS>(Ix + o, vx[0], vx[1], vx[2], vx[3]);
                    store4<TS>(Iy + o, vy[0], vy[1], vy[2], vy[3]);
                }
            } else {
                for (int k = 0; k < 4 && x + k < F.W; ++k) {
                    st(I + o + k, vI[k]);
                    if (F.with_grad) {
                        st(Ix + o + k, vx[k]);
                        st(Iy + o + k, vy[k]);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            d0[k] = d1[k];
            s0[k] = s1[k];
            d1[k] = d2[k];
            s1[k] = s2[k];
            c1[k] = q[k + 1];
        }
    }
    if (!INTERIOR) {  // tiles inside the frame hold no edge pixel; values from the staged bytes
        auto value = [&](int x, int y, float& vI, float& vx, float& vy) {
            const unsigned char* rm = R.row(max(y - 1, 0) - gy0);
            const unsigned char* rc = R.row(y - gy0);
            const unsigned char* rp = R.row(min(y + 1, F.H - 1) - gy0);
            const int xm = max(x - 1, 0) - gx0, xc = x - gx0, xp = min(x + 1, F.W - 1) - gx0;
            const int sx = ((int)rm[xp] - rm[xm]) + 2 * ((int)rc[xp] - rc[xm]) + ((int)rp[xp] - rp[xm]);
            const int sy = ((int)rp[xm] - rm[xm]) + 2 * ((int)rp[xc] - rm[xc]) + ((int)rp[xp] - rm[xp]);
            vI = (float)rc[xc];
            vx = (float)sx * 0.125f;
            vy = (float)sy * 0.125f;
        };
        apron_strips(I, Ix, Iy, F.with_grad, g.pitch, F.W, F.H, X0, Y0, min(X0 + TX, F.W) - 1,
                     min(Y0 + TY, F.H) - 1, value);
    }
}

// Byte offset of level l's region (l >= 1) in the CTA's shared memory: after the
// staged rows and the regions of levels 1 .. l-1.
__host__ __device__ constexpr size_t region_off(int L, int l)
{
    size_t off = round16((size_t)region_pitch(L) * region_h(L));
    for (int k = 1; k < l; ++k) off += round16((size_t)(region_w(L) >> k) * (region_h(L) >> k) * 4);
    return off;
}

// Level l (1 .. L-1) of the tile, then the next: the level's halo'd region as 2x2
// means of the previous one (of the staged bytes at l = 1), then the tile's I, Ix,
// Iy from it. Every region and tile size is a compile-time constant.
template <typename TS, bool INTERIOR, int L, int l, typename ST>
__device__ __forceinline__ void coarse_level(const PyrFrame& F, const LevelGeom* geo, const ST& R,
                                             unsigned char* smem, int X0, int Y0)
{
    constexpr int h = halo(L), TY = tile_h(L);
    constexpr int RW = region_w(L), RH = region_h(L);
    constexpr int rw = RW >> l, rh = RH >> l, pw = RW >> (l - 1);
    constexpr int hl = h >> l;
    const LevelGeom& g = geo[l];
    const int ox = (X0 >> l) - hl, oy = (Y0 >> l) - hl;  // region origin at level l
    float* cur = reinterpret_cast<float*>(smem + region_off(L, l));
    const float* prev = reinterpret_cast<const float*>(smem + region_off(L, l > 1 ? l - 1 : 1));
    // a warp per region row, lanes along it
    const int lane = threadIdx.x & 31;
    for (int ry = threadIdx.x >> 5; ry < rh; ry += kWarps) {
        const bool yin = INTERIOR || (oy + ry >= 0 && oy + ry < g.H);
        float* out = cur + ry * rw;
        if (l == 1) {
            const unsigned char* b0 = R.row(2 * ry);
            const unsigned char* b1 = R.row(2 * ry + 1);
            for (int rx = lane; rx < rw; rx += 32) {
                float v = 0.f;
                if (INTERIOR || (yin && ox + rx >= 0 && ox + rx < g.W))
                    v = (float)(((int)b0[2 * rx] + b0[2 * rx + 1]) + ((int)b1[2 * rx] + b1[2 * rx + 1])) * 0.25f;
                out[rx] = v;
            }
        } else {
            const float* b = prev + (2 * ry) * pw;
            for (int rx = lane; rx < rw; rx += 32) {
                float v = 0.f;
                if (INTERIOR || (yin && ox + rx >= 0 && ox + rx < g.W))
                    v = ((b[2 * rx] + b[2 * rx + 1]) + (b[pw + 2 * rx] + b[pw + 2 * rx + 1])) * 0.25f;
                out[rx] = v;
            }
        }
    }
    __syncthreads();
    TS* I = reinterpret_cast<TS*>(F.base + g.off_I);
    TS* Ix = reinterpret_cast<TS*>(F.base + g.off_Ix);
    TS* Iy = reinterpret_cast<TS*>(F.base + g.off_Iy);
    // outputs by vertical strips: a lane per PX columns (two where the tile row is 64
    // or more wide: pairs stored with one 8- or 4-byte store), a band of rows per
    // lane group
    constexpr int tw = tile_w(L) >> l, th = TY >> l;
    constexpr int PX = tw >= 64 ? 2 : 1;
    constexpr int lanes = tw / PX;  // lanes a row
    constexpr int groups = kThreads / lanes < th ? kThreads / lanes : th;
    constexpr int rs = th / groups;  // rows a band
    const int gi = threadIdx.x / lanes;
    if (gi < groups) {
        const int x = (X0 >> l) + PX * ((int)threadIdx.x % lanes);
        int cx[PX + 2];  // region columns of pixels x-1 .. x+PX, clamped to the level
#pragma unroll
        for (int j = 0; j < PX + 2; ++j) cx[j] = (INTERIOR ? x - 1 + j : min(max(x - 1 + j, 0), g.W - 1)) - ox;
        auto row = [&](int y) { return cur + ((INTERIOR ? y : min(max(y, 0), g.H - 1)) - oy) * rw; };
        const int yb = (Y0 >> l) + gi * rs;
        float a[PX + 2], b[PX + 2];
        {
            const float* r0 = row(yb - 1);
            const float* r1 = row(yb);
#pragma unroll
            for (int j = 0; j < PX + 2; ++j) {
                a[j] = r0[cx[j]];
                b[j] = r1[cx[j]];
            }
        }
        const bool full = INTERIOR || x + PX - 1 < g.W;
#pragma unroll 1
        for (int i = 0; i < rs; ++i) {
            const int y = yb + i;
            const float* r2 = row(y + 1);
            float c[PX + 2];
#pragma unroll
            for (int j = 0; j < PX + 2; ++j) c[j] = r2[cx[j]];
            if (INTERIOR || (x < g.W && y < g.H)) {
                float gx[PX], gy[PX];
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    gx[k] = ((a[k + 2] - a[k]) + 2.f * (b[k + 2] - b[k]) + (c[k + 2] - c[k])) * 0.125f;
                    gy[k] = ((c[k] - a[k]) + 2.f * (c[k + 1] - a[k + 1]) + (c[k + 2] - a[k + 2])) * 0.125f;
                }
                const size_t o = (size_t)y * g.pitch + x;
                if (PX == 2 && full) {
                    store2<TS>(I + o, b[1], b[2]);
                    if (F.with_grad) {
                        store2<TS>(Ix + o, gx[0], gx[PX - 1]);
                        store2<TS>(Iy + o, gy[0], gy[PX - 1]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < PX; ++k) {
                        if (k == 0 || x + k < g.W) {
                            st(I + o + k, b[k + 1]);
                            if (F.with_grad) {
                                st(Ix + o + k, gx[k]);
                                st(Iy + o + k, gy[k]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < PX + 2; ++j) {
                a[j] = b[j];
                b[j] = c[j];
            }
        }
    }
    if (!INTERIOR) {  // values from the level's region in shared memory
        auto value = [&](int x, int y, float& vI, float& vx, float& vy) {
            const int xc = x - ox, yc = y - oy;
            const int xm = max(x - 1, 0) - ox, xp = min(x + 1, g.W - 1) - ox;
            const int ym = max(y - 1, 0) - oy, yp = min(y + 1, g.H - 1) - oy;
            vI = cur[yc * rw + xc];
            const float gx = (cur[ym * rw + xp] - cur[ym * rw + xm]) + 2.f * (cur[yc * rw + xp] - cur[yc * rw + xm]) +
                             (cur[yp * rw + xp] - cur[yp * rw + xm]);
            const float gy = (cur[yp * rw + xm] - cur[ym * rw + xm]) + 2.f * (cur[yp * rw + xc] - cur[ym * rw + xc]) +
                             (cur[yp * rw + xp] - cur[ym * rw + xp]);
            vx = gx * 0.125f;
            vy = gy * 0.125f;
        };
        const int x0 = X0 >> l, y0 = Y0 >> l;
        apron_strips(I, Ix, Iy, F.with_grad, g.pitch, g.W, g.H, x0, y0, min(x0 + tw, g.W) - 1, min(y0 + th, g.H) - 1,
                     value);
    }
    if constexpr (l + 1 < L) coarse_level<TS, INTERIOR, L, l + 1, ST>(F, geo, R, smem, X0, Y0);
}

// Five blocks per SM for up to four levels (48 registers, 8-12 bytes of spills outside
// the row loops): on the 64-pair batch the pyramids took 192 us against 201 us with four
// blocks (64 registers) and 260-276 us with six (40 registers, spills inside the loops);
// at least two beyond.
template <int L>
constexpr int pyramid_min_blocks()
{
    return L <= 4 ? 5 : 2;
}

// Every level of the tile from its staged bytes.
template <typename TS, int L, typename ST>
__device__ __forceinline__ void build_tile(const PyrFrame& F, const LevelGeom* geo, const ST& R, unsigned char* smem,
                                           int X0, int Y0, bool interior)
{
    constexpr int h = halo(L), TY = tile_h(L);
    if (interior) {
        level0<TS, true, tile_w(L), TY>(F, geo[0], R, X0, Y0, h);
        if constexpr (L > 1) coarse_level<TS, true, L, 1>(F, geo, R, smem, X0, Y0);
    } else {
        level0<TS, false, tile_w(L), TY>(F, geo[0], R, X0, Y0, h);
        if constexpr (L > 1) coarse_level<TS, false, L, 1>(F, geo, R, smem, X0, Y0);
    }
}

template <typename TS, int L>
__global__ void __launch_bounds__(kThreads, pyramid_min_blocks<L>()) pyramid_kernel(const __grid_constant__ PyrBatch a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LevelGeom geo[DGF_MAX_LEVELS];
    __shared__ int frame;
    if (threadIdx.x < L) {  // one thread per level: find the frame, then its level geometry
        int f = 0;
        for (int lo = 0, hi = a.n_frames - 1; lo <= hi;) {
            const int mid = (lo + hi) >> 1;
            if (a.frames[mid].cta_begin <= (int)blockIdx.x) {
                f = mid;
                lo = mid + 1;
            } else {
                hi = mid - 1;
            }
        }
        level_geom(a.frames[f].W, a.frames[f].H, L, (int)sizeof(TS), threadIdx.x, &geo[threadIdx.x]);
        if (threadIdx.x == 0) frame = f;
    }
    __syncthreads();
    const PyrFrame& F = a.frames[frame];
    constexpr int h = halo(L), TY = tile_h(L);
    constexpr int RW = region_w(L), RH = region_h(L), RWP = region_pitch(L);
    constexpr int NWR = (RW + 3 + 3) / 4;  // aligned words per row for the word copies (misalignment included)
    const int t = blockIdx.x - F.cta_begin;
    constexpr int TX = tile_w(L);
    const int tiles_x = (F.W + TX - 1) / TX;
    const int X0 = (t % tiles_x) * TX, Y0 = (t / tiles_x) * TY;
    const int gx0 = X0 - h, gy0 = Y0 - h;
    // the halo'd region inside the frame: no clamping at any level
    const bool interior = gx0 >= 0 && gy0 >= 0 && gx0 + RW <= F.W && gy0 + RH <= F.H;

    // 1. stage the frame bytes under the tile and its halo (rows and columns inside the
    // frame; bytes outside it are never read), 2. build every level of the tile
    if (F.bulk) {
        // frame base, pitch and width multiples of 16: one bulk copy per row of the
        // 16-byte aligned span covering the row's columns inside the frame (it stays
        // inside the row), all completing on one barrier
        __shared__ __align__(8) uint64_t bar;
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        const int r_lo = max(gy0, 0) - gy0, r_hi = min(gy0 + RH, F.H) - gy0;
        const int a_lo = max(gx0, 0) & ~15, a_hi = (min(gx0 + RW, F.W) + 15) & ~15;  // frame byte span
        const int base = gx0 & ~15;  // frame column at staged byte 0 of every row
        if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, (unsigned)((r_hi - r_lo) * (a_hi - a_lo)));
        for (int r = r_lo + (int)threadIdx.x; r < r_hi; r += kThreads)
            bulk_copy_to_smem(smem + r * RWP + (a_lo - base), F.img + (long long)(gy0 + r) * F.pitch + a_lo,
                              (unsigned)(a_hi - a_lo), &bar);
        const bool ok = mbar_wait(&bar, 0, kStageWaitTries);
        if (!__syncthreads_and(ok)) {  // the copy engine stopped answering: record, drain, leave
            if (threadIdx.x == 0 && a.status) atomicOr(a.status, (unsigned)DGF_DEV_STAGE_WAIT);
            mbar_wait(&bar, 0, kStageWaitTries);
            return;
        }
        build_tile<TS, L>(F, geo, Staged<L, true>{smem, 0u, 0u}, smem, X0, Y0, interior);
    } else {
        // otherwise every aligned 4-byte word that holds a byte of the region (such a
        // word lies inside the frame's allocation), copied asynchronously
        const long long org = (long long)(uintptr_t)F.img + (long long)gy0 * F.pitch + gx0;
        const Staged<L, false> R{smem, (unsigned)org & 3u, (unsigned)F.pitch & 3u};
        const int cx0 = max(gx0, 0) - gx0, cx1 = min(gx0 + RW, F.W) - gx0;  // region columns inside the frame
        for (int i = threadIdx.x; i < RH * NWR; i += kThreads) {
            const int r = i / NWR, k = i - r * NWR;
            const int gy = gy0 + r;
            const int c_lo = 4 * k - (int)((R.mis0 + (unsigned)r * R.pmod) & 3u);  // region column of the word's first byte
            if (gy < 0 || gy >= F.H || c_lo + 3 < cx0 || c_lo >= cx1) continue;
            cp_async4(smem + r * RWP + 4 * k, F.img + (long long)gy * F.pitch + gx0 + c_lo);
        }
        cp_async_wait_all();
        __syncthreads();
        build_tile<TS, L>(F, geo, R, smem, X0, Y0, interior);
    }
}

// Fills the CTA prefix counts and launches one pyramid build for every frame.
int launch_pyramids(PyrBatch& a, int storage, cudaStream_t stream)
{
    long long ctas = 0;
    for (int f = 0; f < a.n_frames; ++f) {
        PyrFrame& F = a.frames[f];
        F.cta_begin = (int)ctas;
        // rows whose 16-byte spans end at or before the row's last byte: no copy reads
        // past the frame, whatever lies beyond its last row
        F.bulk = aligned(F.img, 16) && F.pitch % 16 == 0 && F.W % 16 == 0;
        ctas += frame_ctas(F.W, F.H, a.levels);
    }
    a.status = status_word();
    if (ctas == 0) return DGF_OK;
    if (ctas > 0x7fffffffLL) return DGF_ERR_ARG;
    const size_t smem = smem_bytes(a.levels);
    const unsigned grid = (unsigned)ctas;
#define DGF_PYR(L)                                                                           \
    case L:                                                                                  \
        if (storage == DGF_F32)                                                              \
            pyramid_kernel<float, L><<<grid, kThreads, smem, stream>>>(a);                  \
        else                                                                                 \
            pyramid_kernel<__half, L><<<grid, kThreads, smem, stream>>>(a);                 \
        break;
    switch (a.levels) {
        DGF_PYR(1)
        DGF_PYR(2)
        DGF_PYR(3)
        DGF_PYR(4)
        DGF_PYR(5)
        DGF_PYR(6)
        default:
            return DGF_ERR_ARG;
    }
#undef DGF_PYR
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
