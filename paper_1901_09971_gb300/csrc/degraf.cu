// DeGraF key-point detection (arXiv 1901.09971, Section 2, Eq. 1-2).
//
// One thread per window. A CTA covers 32 x BY windows; when they overlap
// (step < window) the union of their pixels is staged once in shared memory,
// otherwise each thread reads its window straight from global memory. The window
// sums S = sum I, X = sum j I, Y = sum i I and the maximum m are exact int32; the
// negative-centroid sums follow from them in closed form,
//   S_neg = n (1+m) - S,  X_neg = (1+m) h w (w-1)/2 - X,  Y_neg = (1+m) w h (h-1)/2 - Y,
// and the selected centroid is formed in FP64 and rounded once to FP32, so every
// coordinate is the exactly rounded value of Eq. 1 or Eq. 2 plus the window origin.
#include "common.cuh"

namespace {

constexpr int kBX = 32;

struct DetectArgs {
    const uint8_t* img;
    int W, H, pitch, ww, wh, step, nu, nv;
    float* pts;
    int32_t* sums;
};

__device__ __forceinline__ void emit(const DetectArgs& a, int u, int v, int S, int X, int Y, int m)
{
    const int n = a.ww * a.wh;
    const int m1 = m + 1;
    const int Sn = n * m1 - S;
    double cx, cy;
    if (Sn > S) {  // Eq. 2 centroid: the larger weight sum wins, ties keep C_pos
        const int Xn = m1 * (a.wh * (a.ww * (a.ww - 1) / 2)) - X;
        const int Yn = m1 * (a.ww * (a.wh * (a.wh - 1) / 2)) - Y;
        cx = (double)Xn / (double)Sn;
        cy = (double)Yn / (double)Sn;
    } else {  // Eq. 1 centroid
        cx = (double)X / (double)S;
        cy = (double)Y / (double)S;
    }
    const long long k = (long long)v * a.nu + u;
    const float2 p = make_float2((float)((double)(u * a.step) + cx), (float)((double)(v * a.step) + cy));
    reinterpret_cast<float2*>(a.pts)[k] = p;
    if (a.sums) reinterpret_cast<int4*>(a.sums)[k] = make_int4(S, X, Y, m);
}

template <bool kStaged>
__global__ void __launch_bounds__(256) degraf_detect_kernel(DetectArgs a, int tile_w, int tile_h)
{
    extern __shared__ uint8_t tile[];
    const int u0 = blockIdx.x * kBX, v0 = blockIdx.y * blockDim.y;
    const int x0 = u0 * a.step, y0 = v0 * a.step;
    if (kStaged) {
        const int tw = min(tile_w, a.W - x0), th = min(tile_h, a.H - y0);
        for (int r = threadIdx.y; r < th; r += blockDim.y) {
            const uint8_t* src = a.img + (size_t)(y0 + r) * a.pitch + x0;
            for (int c = threadIdx.x; c < tw; c += blockDim.x) tile[r * tile_w + c] = src[c];
        }
        __syncthreads();
    }
    const int u = u0 + threadIdx.x, v = v0 + threadIdx.y;
    if (u >= a.nu || v >= a.nv) return;
    const uint8_t* w0;
    int rstride;
    if (kStaged) {
        w0 = tile + threadIdx.y * a.step * tile_w + threadIdx.x * a.step;
        rstride = tile_w;
    } else {
        w0 = a.img + (size_t)(v * a.step) * a.pitch + u * a.step;
        rstride = a.pitch;
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
    emit(a, u, v, S, X, Y, m);
}

long long grid_count(int n, int win, int step) { return n < win ? 0 : (long long)((n - win) / step) + 1; }

}  // namespace

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
    if (!pts || !dgf::aligned(pts, 8) || (sums && !dgf::aligned(sums, 16))) return DGF_ERR_ARG;
    DetectArgs a{img, W, H, pitch, win_w, win_h, step, (int)grid_count(W, win_w, step),
                 (int)grid_count(H, win_h, step), pts, sums};
    const bool overlap = step < win_w || step < win_h;
    int by = 8;
    int tile_w = (kBX - 1) * step + win_w;
    int tile_h = (by - 1) * step + win_h;
    const int kSmemMax = 48 * 1024;
    while (by > 1 && tile_w * tile_h > kSmemMax) {
        by /= 2;
        tile_h = (by - 1) * step + win_h;
    }
    const bool staged = overlap && tile_w * tile_h <= kSmemMax;
    dim3 block(kBX, by);
    dim3 grid((a.nu + kBX - 1) / kBX, (a.nv + by - 1) / by);
    if (grid.y > 65535) return DGF_ERR_ARG;
    if (staged)
        degraf_detect_kernel<true><<<grid, block, (size_t)tile_w * tile_h, stream>>>(a, tile_w, tile_h);
    else
        degraf_detect_kernel<false><<<grid, block, 0, stream>>>(a, 0, 0);
    return dgf::launch_status();
}
