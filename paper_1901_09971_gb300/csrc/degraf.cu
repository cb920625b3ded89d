// DeGraF key-point detection (arXiv 1901.09971, Section 2, Eq. 1-2).
//
// One thread per window. A CTA covers 32 x BY windows of one frame (a launch may
// cover the frames of a whole batch); when they overlap (step < window) the union
// of their pixels is staged once in shared memory, otherwise each thread reads its
// window straight from global memory. The window
// sums S = sum I, X = sum j I, Y = sum i I and the maximum m are exact int32; the
// negative-centroid sums follow from them in closed form,
//   S_neg = n (1+m) - S,  X_neg = (1+m) h w (w-1)/2 - X,  Y_neg = (1+m) w h (h-1)/2 - Y,
// and the selected centroid is formed in FP64 and rounded once to FP32, so every
// coordinate is the exactly rounded value of Eq. 1 or Eq. 2 plus the window origin.
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
    double cx, cy;
    if (Sn > S) {  // Eq. 2 centroid: the larger weight sum wins, ties keep C_pos
        const int Xn = m1 * (wh * (ww * (ww - 1) / 2)) - X;
        const int Yn = m1 * (ww * (wh * (wh - 1) / 2)) - Y;
        cx = (double)Xn / (double)Sn;
        cy = (double)Yn / (double)Sn;
    } else {  // Eq. 1 centroid
        cx = (double)X / (double)S;
        cy = (double)Y / (double)S;
    }
    const long long k = (long long)v * J.nu + u;
    reinterpret_cast<float2*>(J.pts)[k] =
        make_float2((float)((double)(u * J.step) + cx), (float)((double)(v * J.step) + cy));
    if (J.sums) reinterpret_cast<int4*>(J.sums)[k] = make_int4(S, X, Y, m);
}

// One thread per window; CTAs of all frames of the batch in one grid.
__global__ void __launch_bounds__(256) degraf_detect_kernel(const __grid_constant__ DetectBatch a)
{
    extern __shared__ uint8_t tile[];
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
    if (a.staged) {
        const int tw = min(tile_w, J.W - x0), th = min(tile_h, J.H - y0);
        for (int r = threadIdx.y; r < th; r += blockDim.y) {
            const uint8_t* src = J.img + (size_t)(y0 + r) * J.pitch + x0;
            for (int c = threadIdx.x; c < tw; c += blockDim.x) tile[r * tile_w + c] = src[c];
        }
        __syncthreads();
    }
    const int u = u0 + threadIdx.x, v = v0 + threadIdx.y;
    if (u >= J.nu || v >= J.nv) return;
    const uint8_t* w0;
    int rstride;
    if (a.staged) {
        w0 = tile + threadIdx.y * J.step * tile_w + threadIdx.x * J.step;
        rstride = tile_w;
    } else {
        w0 = J.img + (size_t)(v * J.step) * J.pitch + u * J.step;
        rstride = J.pitch;
    }
    int S = 0, X = 0, Y = 0, m = 0;
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
    const int tile_w = (kBX - 1) * max_step + a.ww;
    int tile_h = (by - 1) * max_step + a.wh;
    while (by > 1 && tile_w * tile_h > kSmemMax) {
        by /= 2;
        tile_h = (by - 1) * max_step + a.wh;
    }
    a.by = by;
    a.staged = overlap && tile_w * tile_h <= kSmemMax;
    a.tile_w = tile_w;
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
