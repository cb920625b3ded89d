// Image pyramid with Sobel gradients for RLOF tracking (arXiv 1901.09971, Section 2,
// "Sparse point tracking": RLOF works coarse to fine over an image pyramid that the
// paper does not define).
//
// Definition used: level l+1 = 2x2 block means of level l (sizes floor(W_l/2) x
// floor(H_l/2)); Ix, Iy = Sobel / 8 with clamped borders. Every level value is an
// integer byte sum times 4^-l and every Sobel sum a small multiple of it, so all of
// them are exact in FP32 (FP16 storage rounds each exact value once).
//
// One CTA owns a 64 x TY tile of level 0 (TY = 128 for up to 4 levels, 32 beyond)
// and produces the matching tile of every level. It stages the frame bytes under
// the tile plus a halo of 2^(L-1) pixels (enough for a one-pixel halo at the
// coarsest level) with asynchronous 4-byte copies (cp.async) of the aligned words
// that hold them: frame rows need not start on any boundary, so each staged row
// keeps its own misalignment (0..3 bytes) and every read adds it. Then the CTA walks
// down the levels, forming each level's values on its halo'd region from the
// previous one with 2x2 means and writing I, Ix, Iy of the tile with coalesced rows
// (16-byte stores at level 0). Tiles on the frame's edge also write the planes'
// replicated borders (kApron pixels wide; the clamped values, so that tracking reads
// its taps without clamping). Tall tiles mean few staging round trips per SM; the
// frame is read about once from DRAM and every output byte is written once.
#include "common.cuh"
#include "batch.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kTX = 64;  // level-0 tile width

__host__ __device__ constexpr int tile_h(int levels) { return levels <= 4 ? 128 : 32; }
__host__ __device__ constexpr int halo(int levels) { return levels >= 2 ? 1 << (levels - 1) : 1; }
__host__ __device__ constexpr int region_w(int levels) { return kTX + 2 * halo(levels); }
__host__ __device__ constexpr int region_h(int levels) { return tile_h(levels) + 2 * halo(levels); }
// staged row pitch: the region's bytes plus up to 15 bytes of row offset on either
// side (bulk copies move 16-byte-aligned spans), a multiple of 16
__host__ __device__ constexpr int region_pitch(int levels) { return (region_w(levels) + 32 + 15) & ~15; }

__host__ __device__ inline int frame_ctas(int W, int H, int levels)
{
    return ((W + kTX - 1) / kTX) * ((H + tile_h(levels) - 1) / tile_h(levels));
}

__host__ __device__ inline size_t round16(size_t v) { return (v + 15) & ~(size_t)15; }

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

// Staged region rows: byte (r, c) of the halo'd region (frame pixel (gx0 + c,
// gy0 + r)) sits at raw[r * RWP + mis(r) + c]. Word copies: mis(r) is the
// misalignment of that frame row's byte gx0 (rows advance by the pitch, so it steps
// by pitch mod 4, mask 3). Bulk copies: every row has the same offset, gx0 mod 16.
struct Staged {
    const unsigned char* raw;
    unsigned mis0, pmod, mask;
    int RWP;
    __device__ __forceinline__ const unsigned char* row(int r) const
    {
        return raw + r * RWP + ((mis0 + (unsigned)r * pmod) & mask);
    }
};

}  // namespace

namespace dgf {

// The replicated border (kApron pixels wide) that a tile on a level's edge owns:
// outside the level, beside the tile's columns [x0, xe] and rows [y0, ye] (its part
// of the level), every position takes the values at its clamped position, which
// lies in the tile. The left and right strips include the corner blocks. All
// threads of the block share the strips; value(x, y, I, Ix, Iy) forms the values of
// tile pixel (x, y) from the data the block already holds.
template <typename TS, typename Value>
__device__ __forceinline__ void apron_strips(TS* I, TS* Ix, TS* Iy, bool grad, int pitch, int W, int H, int x0,
                                             int y0, int xe, int ye, Value value)
{
    if (xe < x0 || ye < y0) return;  // the tile holds no pixel of this level
    const bool L = x0 == 0, R = xe == W - 1, T = y0 == 0, B = ye == H - 1;
    if (!(L || R || T || B)) return;
    const int ry0 = T ? -kApron : y0, ry1 = B ? H - 1 + kApron : ye;  // rows of the side strips
    const int sh = ry1 - ry0 + 1, tw = xe - x0 + 1;
    auto put = [&](int ax, int ay) {
        float vI, vx, vy;
        value(min(max(ax, 0), W - 1), min(max(ay, 0), H - 1), vI, vx, vy);
        const ptrdiff_t o = (ptrdiff_t)ay * pitch + ax;
        st(I + o, vI);
        if (grad) {
            st(Ix + o, vx);
            st(Iy + o, vy);
        }
    };
    if (L)
        for (int i = threadIdx.x; i < kApron * sh; i += blockDim.x) put(i % kApron - kApron, ry0 + i / kApron);
    if (R)
        for (int i = threadIdx.x; i < kApron * sh; i += blockDim.x) put(W + i % kApron, ry0 + i / kApron);
    if (T)
        for (int i = threadIdx.x; i < kApron * tw; i += blockDim.x) put(x0 + i % tw, i / tw - kApron);
    if (B)
        for (int i = threadIdx.x; i < kApron * tw; i += blockDim.x) put(x0 + i % tw, H + i / tw);
}

// Level 0 of the tile: I and Sobel / 8 straight from the staged bytes, four
// pixels per item. INTERIOR: the halo'd region lies inside the frame, so no
// neighbour needs clamping.
template <typename TS, bool INTERIOR, int TY>
__device__ __forceinline__ void level0(const PyrFrame& F, const LevelGeom& g, const Staged& R, int X0, int Y0, int h)
{
    TS* I = reinterpret_cast<TS*>(F.base + g.off_I);
    TS* Ix = reinterpret_cast<TS*>(F.base + g.off_Ix);
    TS* Iy = reinterpret_cast<TS*>(F.base + g.off_Iy);
    const int gx0 = X0 - h, gy0 = Y0 - h;
    for (int i = threadIdx.x; i < TY * (kTX / 4); i += blockDim.x) {
        const int ty = i >> 4, tx = (i & 15) << 2;  // kTX / 4 = 16 items per row
        const int y = Y0 + ty;
        if (!INTERIOR && (y >= F.H || X0 + tx >= F.W)) continue;
        float vI[4], vx[4], vy[4];
        if (INTERIOR) {
            const unsigned char* rm = R.row(ty + h - 1) + tx + h - 1;  // columns x-1 .. x+4
            const unsigned char* rc = R.row(ty + h) + tx + h - 1;
            const unsigned char* rp = R.row(ty + h + 1) + tx + h - 1;
            int a[6], b[6], c[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                a[j] = rm[j];
                b[j] = rc[j];
                c[j] = rp[j];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int sx = (a[k + 2] - a[k]) + 2 * (b[k + 2] - b[k]) + (c[k + 2] - c[k]);
                const int sy = (c[k] - a[k]) + 2 * (c[k + 1] - a[k + 1]) + (c[k + 2] - a[k + 2]);
                vI[k] = (float)b[k + 1];
                vx[k] = (float)sx * 0.125f;
                vy[k] = (float)sy * 0.125f;
            }
        } else {
            const unsigned char* rm = R.row(max(y - 1, 0) - gy0);
            const unsigned char* rc = R.row(y - gy0);
            const unsigned char* rp = R.row(min(y + 1, F.H - 1) - gy0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = min(X0 + tx + k, F.W - 1);  // past the edge: recomputed, not stored
                const int xm = max(x - 1, 0) - gx0, xc = x - gx0, xp = min(x + 1, F.W - 1) - gx0;
                const int sx = ((int)rm[xp] - rm[xm]) + 2 * ((int)rc[xp] - rc[xm]) + ((int)rp[xp] - rp[xm]);
                const int sy = ((int)rp[xm] - rm[xm]) + 2 * ((int)rp[xc] - rm[xc]) + ((int)rp[xp] - rm[xp]);
                vI[k] = (float)rc[xc];
                vx[k] = (float)sx * 0.125f;
                vy[k] = (float)sy * 0.125f;
            }
        }
        const size_t o = (size_t)y * g.pitch + X0 + tx;
        if (INTERIOR || X0 + tx + 3 < F.W) {
            store4<TS>(I + o, vI[0], vI[1], vI[2], vI[3]);
            if (F.with_grad) {
                store4<TS>(Ix + o, vx[0], vx[1], vx[2], vx[3]);
                store4<TS>(Iy + o, vy[0], vy[1], vy[2], vy[3]);
            }
        } else {
            for (int k = 0; k < 4 && X0 + tx + k < F.W; ++k) {
                st(I + o + k, vI[k]);
                if (F.with_grad) {
                    st(Ix + o + k, vx[k]);
                    st(Iy + o + k, vy[k]);
                }
            }
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
        apron_strips(I, Ix, Iy, F.with_grad, g.pitch, F.W, F.H, X0, Y0, min(X0 + kTX, F.W) - 1,
                     min(Y0 + TY, F.H) - 1, value);
    }
}

// Levels 1 .. L-1 of the tile: each level's halo'd region as 2x2 means of the
// previous one, then the tile's I, Ix, Iy from it. The level loop unrolls, so every
// region size is a compile-time constant (flat loops, constant divisors).
template <typename TS, bool INTERIOR, int L>
__device__ __forceinline__ void coarse_levels(const PyrFrame& F, const LevelGeom* geo, const Staged& R,
                                              unsigned char* smem, int X0, int Y0)
{
    constexpr int h = halo(L), TY = tile_h(L);
    constexpr int RW = region_w(L), RH = region_h(L);
    size_t prev_off = 0, cur_off = round16((size_t)region_pitch(L) * RH);
#pragma unroll
    for (int l = 1; l < L; ++l) {
        if (l > 1) {
            prev_off = cur_off;
            cur_off += round16((size_t)(RW >> (l - 1)) * (RH >> (l - 1)) * 4);
        }
        const LevelGeom& g = geo[l];
        const int rw = RW >> l, rh = RH >> l, pw = RW >> (l - 1);
        const int hl = h >> l;
        const int ox = (X0 >> l) - hl, oy = (Y0 >> l) - hl;  // region origin at level l
        float* cur = reinterpret_cast<float*>(smem + cur_off);
        const float* prev = reinterpret_cast<const float*>(smem + prev_off);
        for (int i = threadIdx.x; i < rw * rh; i += kThreads) {
            const int ry = i / rw, rx = i - ry * rw;
            float v = 0.f;
            if (INTERIOR || (ox + rx >= 0 && ox + rx < g.W && oy + ry >= 0 && oy + ry < g.H)) {
                if (l == 1) {
                    const unsigned char* b0 = R.row(2 * ry) + 2 * rx;
                    const unsigned char* b1 = R.row(2 * ry + 1) + 2 * rx;
                    v = (float)(((int)b0[0] + b0[1]) + ((int)b1[0] + b1[1])) * 0.25f;
                } else {
                    const float* b = prev + (2 * ry) * pw + 2 * rx;
                    v = ((b[0] + b[1]) + (b[pw] + b[pw + 1])) * 0.25f;
                }
            }
            cur[i] = v;
        }
        __syncthreads();
        TS* I = reinterpret_cast<TS*>(F.base + g.off_I);
        TS* Ix = reinterpret_cast<TS*>(F.base + g.off_Ix);
        TS* Iy = reinterpret_cast<TS*>(F.base + g.off_Iy);
        const int tw = kTX >> l, th = TY >> l;
        for (int i = threadIdx.x; i < tw * th; i += kThreads) {
            const int ty = i / tw, tx = i - ty * tw;
            const int x = (X0 >> l) + tx, y = (Y0 >> l) + ty;
            if (!INTERIOR && (x >= g.W || y >= g.H)) continue;
            const int xc = tx + hl, yc = ty + hl;
            const int xm = INTERIOR ? xc - 1 : max(x - 1, 0) - ox, xp = INTERIOR ? xc + 1 : min(x + 1, g.W - 1) - ox;
            const int ym = INTERIOR ? yc - 1 : max(y - 1, 0) - oy, yp = INTERIOR ? yc + 1 : min(y + 1, g.H - 1) - oy;
            const size_t o = (size_t)y * g.pitch + x;
            const float v = cur[yc * rw + xc];
            st(I + o, v);
            if (F.with_grad) {
                const float gx = (cur[ym * rw + xp] - cur[ym * rw + xm]) + 2.f * (cur[yc * rw + xp] - cur[yc * rw + xm]) +
                                 (cur[yp * rw + xp] - cur[yp * rw + xm]);
                const float gy = (cur[yp * rw + xm] - cur[ym * rw + xm]) + 2.f * (cur[yp * rw + xc] - cur[ym * rw + xc]) +
                                 (cur[yp * rw + xp] - cur[ym * rw + xp]);
                st(Ix + o, gx * 0.125f);
                st(Iy + o, gy * 0.125f);
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
            apron_strips(I, Ix, Iy, F.with_grad, g.pitch, g.W, g.H, x0, y0, min(x0 + tw, g.W) - 1,
                         min(y0 + th, g.H) - 1, value);
        }
    }
}

// Six blocks per SM for up to four levels (tall tiles, 40 registers: measured 2.4% faster on the
// 64-pair batch than four blocks at 64 registers, eight blocks at 32 spill and lose), at least
// two beyond.
template <int L>
constexpr int pyramid_min_blocks()
{
    return L <= 4 ? 6 : 2;
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
    const int tiles_x = (F.W + kTX - 1) / kTX;
    const int X0 = (t % tiles_x) * kTX, Y0 = (t / tiles_x) * TY;
    const int gx0 = X0 - h, gy0 = Y0 - h;
    // the halo'd region inside the frame: no clamping at any level
    const bool interior = gx0 >= 0 && gy0 >= 0 && gx0 + RW <= F.W && gy0 + RH <= F.H;

    // 1. stage the frame bytes under the tile and its halo (rows and columns inside the
    // frame; bytes outside it are never read)
    Staged R;
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
        R = Staged{smem, (unsigned)(gx0 - base), 0u, 15u, RWP};
    } else {
        // otherwise every aligned 4-byte word that holds a byte of the region (such a
        // word lies inside the frame's allocation), copied asynchronously
        const long long org = (long long)(uintptr_t)F.img + (long long)gy0 * F.pitch + gx0;
        R = Staged{smem, (unsigned)org & 3u, (unsigned)F.pitch & 3u, 3u, RWP};
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
    }

    if (interior) {
        level0<TS, true, TY>(F, geo[0], R, X0, Y0, h);
        coarse_levels<TS, true, L>(F, geo, R, smem, X0, Y0);
    } else {
        level0<TS, false, TY>(F, geo[0], R, X0, Y0, h);
        coarse_levels<TS, false, L>(F, geo, R, smem, X0, Y0);
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
