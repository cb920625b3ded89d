// DeGraF key-point detection (arXiv 1901.09971, Section 2, Eq. 1-2).
//
// One thread per window. A CTA covers 32 x BY windows of one frame (a launch may
// cover the frames of a whole batch); when they overlap (step < window) the union
// of their pixels is staged once in shared memory, otherwise each thread reads its
// window straight from global memory. The window
// sums S = sum I, X = sum j I, Y = sum i I and the maximum m are exact int32; the
// negative-centroid sums follow from them in closed form,
//   S_neg = n (1+m) - S,  X_neg = (1+m) h w (w-1)/2 - X,  Y_neg = (1+m) w h (h-1)/2 - Y,
// and the selected centroid is an FP32 quotient of exact integers plus the window
// origin (two correctly rounded steps, within one FP32 ulp of Eq. 1 or Eq. 2).
#include "common.cuh"
#include "batch.cuh"

namespace {

constexpr int kBX = 32;       // windows per CTA along x
constexpr int kSmemMax = 48 * 1024;

long long grid_count(int n, int win, int step) { return n < win ? 0 : (long long)((n - win) / step) + 1; }

}  // namespace

namespace dgf {

__device__ __forceinline__ void emit(const DetectJob& J, int ww, int wh, int u, int v, int S, int X, int Y, int m)
{
    const int n = ww * wh;
    const int m1 = m + 1;
    const int Sn = n * m1 - S;
    int num_x, num_y, den;
    if (Sn > S) {  // Eq. 2 centroid: the larger weight sum wins, ties keep C_pos
        num_x = m1 * (wh * (ww * (ww - 1) / 2)) - X;
        num_y = m1 * (ww * (wh * (wh - 1) / 2)) - Y;
        den = Sn;
    } else {  // Eq. 1 centroid
        num_x = X;
        num_y = Y;
        den = S;
    }
    // correctly rounded quotients, then the window origin: one rounding each. FP32
    // operands are exact below 2^24 (every window up to about 45 x 45); larger
    // moments divide in FP64 (GB300's FP64 rate is low, so only where needed)
    float cx, cy;
    if (num_x < (1 << 24) && num_y < (1 << 24) && den < (1 << 24)) {
        cx = __fdiv_rn((float)num_x, (float)den);
        cy = __fdiv_rn((float)num_y, (float)den);
    } else {
        cx = (float)((double)num_x / (double)den);
        cy = (float)((double)num_y / (double)den);
    }
    const long long k = (long long)v * J.nu + u;
    reinterpret_cast<float2*>(J.pts)[k] = make_float2(__fadd_rn((float)(u * J.step), cx), __fadd_rn((float)(v * J.step), cy));
    if (J.sums) reinterpret_cast<int4*>(J.sums)[k] = make_int4(S, X, Y, m);
}

// Window sums of a window of width <= 8 from a staged tile whose rows start on
// 4-byte boundaries: per row, the window's bytes become two 32-bit words (funnel
// shifts of three aligned loads), bytes past the window are masked off, and
// dp4a forms the row sum and the column-weighted row sum while a bytewise max
// tracks m.
__device__ __forceinline__ void window_sums_packed(const uint8_t* tile, int stride, int c0, int r0, int ww, int wh,
                                                   int& S, int& X, int& Y, int& m)
{
    const unsigned shift = (c0 & 3) * 8;
    const unsigned mlo = ww >= 4 ? 0xffffffffu : (1u << (8 * ww)) - 1u;
    const unsigned mhi = ww >= 8 ? 0xffffffffu : ww <= 4 ? 0u : (1u << (8 * (ww - 4))) - 1u;
    const unsigned* row = reinterpret_cast<const unsigned*>(tile + r0 * stride) + (c0 >> 2);
    unsigned mx = 0;
    int s = 0, x = 0, y = 0;
    for (int i = 0; i < wh; ++i) {
        const unsigned w0 = row[0], w1 = row[1], w2 = row[2];
        const unsigned lo = __funnelshift_r(w0, w1, shift) & mlo;
        const unsigned hi = __funnelshift_r(w1, w2, shift) & mhi;
        const int rs = (int)__dp4a(lo, 0x01010101u, __dp4a(hi, 0x01010101u, 0u));
        x += (int)__dp4a(lo, 0x03020100u, __dp4a(hi, 0x07060504u, 0u));
        s += rs;
        y += i * rs;
        mx = __vmaxu4(mx, __vmaxu4(lo, hi));
        row += stride >> 2;
    }
    mx = __vmaxu4(mx, mx >> 16);
    mx = __vmaxu4(mx, mx >> 8);
    S = s;
    X = x;
    Y = y;
    m = (int)(mx & 0xffu);
}

// One thread per window; CTAs of all frames of the batch in one grid.
__global__ void __launch_bounds__(256) degraf_detect_kernel(const __grid_constant__ DetectBatch a)
{
    extern __shared__ __align__(16) uint8_t tile[];
    int f = 0;
    for (int lo = 0, hi = a.n_jobs - 1; lo <= hi;) {
        const int mid = (lo + hi) >> 1;
        if (a.jobs[mid].cta_begin <= (int)blockIdx.x) {
            f = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    const DetectJob& J = a.jobs[f];
    const int t = blockIdx.x - J.cta_begin;
    const int u0 = (t % J.tiles_x) * kBX, v0 = (t / J.tiles_x) * blockDim.y;
    const int x0 = u0 * J.step, y0 = v0 * J.step;
    const int tile_w = (kBX - 1) * J.step + a.ww, tile_h = ((int)blockDim.y - 1) * J.step + a.wh;
    const int stride = a.tile_w;  // row stride of the staged tile (multiple of 4)
    if (a.staged) {
        // stage the pixels under the CTA's windows as aligned 32-bit words: per row
        // the word under each 4-byte group and, for a misaligned row, the next word
        // (only if it still holds a byte of the tile, so no load leaves the frame),
        // funnel-shifted; 4 rows x 2 words per thread in flight at a time
        const int tw = min(tile_w, J.W - x0), th = min(tile_h, J.H - y0);
        const int nw = (tw + 3) >> 2;
        unsigned* tile32 = reinterpret_cast<unsigned*>(tile);
        for (int r0 = threadIdx.y; r0 < th; r0 += 4 * blockDim.y) {
            unsigned lo[4][2], hi[4][2], sh[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = r0 + i * blockDim.y;
                const uintptr_t src = reinterpret_cast<uintptr_t>(J.img + (size_t)(y0 + min(r, th - 1)) * J.pitch + x0);
                const unsigned a = (unsigned)(src & 3u);
                const unsigned* w = reinterpret_cast<const unsigned*>(src & ~(uintptr_t)3);
                sh[i] = a * 8u;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int k = threadIdx.x + 32 * m;
                    const bool ok = r < th && k < nw;
                    lo[i][m] = ok ? __ldg(w + k) : 0u;
                    hi[i][m] = ok && a && 4 * (k + 1) - (int)a < tw ? __ldg(w + k + 1) : 0u;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = r0 + i * blockDim.y;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int k = threadIdx.x + 32 * m;
                    if (r < th && k < nw) tile32[r * (stride >> 2) + k] = __funnelshift_r(lo[i][m], hi[i][m], sh[i]);
                }
            }
        }
        for (int k = 64 + threadIdx.x; k < nw; k += 32)  // rows wider than 256 bytes (large steps)
            for (int r = threadIdx.y; r < th; r += blockDim.y) {
                const uintptr_t src = reinterpret_cast<uintptr_t>(J.img + (size_t)(y0 + r) * J.pitch + x0);
                const unsigned a = (unsigned)(src & 3u);
                const unsigned* w = reinterpret_cast<const unsigned*>(src & ~(uintptr_t)3);
                const unsigned lo = __ldg(w + k), hi = a && 4 * (k + 1) - (int)a < tw ? __ldg(w + k + 1) : 0u;
                tile32[r * (stride >> 2) + k] = __funnelshift_r(lo, hi, a * 8u);
            }
        __syncthreads();
    }
    const int u = u0 + threadIdx.x, v = v0 + threadIdx.y;
    if (u >= J.nu || v >= J.nv) return;
    int S = 0, X = 0, Y = 0, m = 0;
    if (a.staged && a.ww <= 8) {
        window_sums_packed(tile, stride, threadIdx.x * J.step, threadIdx.y * J.step, a.ww, a.wh, S, X, Y, m);
    } else {
        const uint8_t* w0;
        int rstride;
        if (a.staged) {
            w0 = tile + threadIdx.y * J.step * stride + threadIdx.x * J.step;
            rstride = stride;
        } else {
            w0 = J.img + (size_t)(v * J.step) * J.pitch + u * J.step;
            rstride = J.pitch;
        }
        for (int i = 0; i < a.wh; ++i) {
            const uint8_t* row = w0 + (size_t)i * rstride;
            int rs = 0, rx = 0;
            for (int j = 0; j < a.ww; ++j) {
                const int I = row[j];
                rs += I;
                rx += j * I;
                m = max(m, I);
            }
            S += rs;
            X += rx;
            Y += i * rs;
        }
    }
    emit(J, a.ww, a.wh, u, v, S, X, Y, m);
}

// Chooses the CTA shape (32 x by windows, staged through shared memory when the
// windows overlap and every frame's tile fits), fills the CTA prefix counts and
// launches detection for every frame of the batch.
int launch_detect(DetectBatch& a, cudaStream_t stream)
{
    int max_step = 1;
    bool overlap = true;
    for (int f = 0; f < a.n_jobs; ++f) {
        max_step = a.jobs[f].step > max_step ? a.jobs[f].step : max_step;
        overlap = overlap && (a.jobs[f].step < a.ww || a.jobs[f].step < a.wh);
    }
    int by = 8;
    // rows padded to 4 bytes plus two words, so the packed path's three aligned
    // word loads past a window start stay inside the row
    const int tile_w = ((kBX - 1) * max_step + a.ww + 3) / 4 * 4 + 8;
    int tile_h = (by - 1) * max_step + a.wh;
    while (by > 1 && tile_w * tile_h > kSmemMax) {
        by /= 2;
        tile_h = (by - 1) * max_step + a.wh;
    }
    a.by = by;
    a.staged = overlap && tile_w * tile_h <= kSmemMax;
    a.tile_w = tile_w;  // row stride of the staged tile
    a.tile_h = tile_h;
    long long ctas = 0;
    for (int f = 0; f < a.n_jobs; ++f) {
        DetectJob& J = a.jobs[f];
        J.tiles_x = (J.nu + kBX - 1) / kBX;
        J.cta_begin = (int)ctas;
        ctas += (long long)J.tiles_x * ((J.nv + by - 1) / by);
    }
    if (ctas == 0) return DGF_OK;
    if (ctas > 0x7fffffffLL) return DGF_ERR_ARG;
    degraf_detect_kernel<<<(unsigned)ctas, dim3(kBX, by), a.staged ? (size_t)tile_w * tile_h : 0, stream>>>(a);
    return launch_status();
}

}  // namespace dgf

extern "C" long long dgf_degraf_count(int W, int H, int win_w, int win_h, int step)
{
    if (W < 1 || H < 1 || win_w < 1 || win_h < 1 || win_w > DGF_MAX_WINDOW || win_h > DGF_MAX_WINDOW ||
        step < 1)
        return -1;
    return grid_count(W, win_w, step) * grid_count(H, win_h, step);
}

extern "C" int degraf_detect(const uint8_t* img, int W, int H, int pitch, int win_w, int win_h, int step,
                             float* pts, int32_t* sums, cudaStream_t stream)
{
    const long long n = dgf_degraf_count(W, H, win_w, win_h, step);
    if (n < 0 || !img || pitch < W) return DGF_ERR_ARG;
    if (n == 0) return DGF_OK;
    if (!pts || !dgf::aligned(pts, 8) || (sums && !dgf::aligned(sums, 16)) || n > 0x7fffffffLL) return DGF_ERR_ARG;
    dgf::DetectBatch a = {};
    a.ww = win_w;
    a.wh = win_h;
    a.n_jobs = 1;
    dgf::DetectJob& J = a.jobs[0];
    J.img = img;
    J.W = W;
    J.H = H;
    J.pitch = pitch;
    J.step = step;
    J.nu = (int)grid_count(W, win_w, step);
    J.nv = (int)grid_count(H, win_h, step);
    J.pts = pts;
    J.sums = sums;
    return dgf::launch_detect(a, stream);
}
