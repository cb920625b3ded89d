// DeGraF key-point detection (arXiv 1901.09971, Section 2, Eq. 1-2).
//
// One thread per window column and vr (4) consecutive windows along it; a CTA covers
// 32 x (by vr) windows of one frame (a launch may cover the frames of a whole batch).
// When windows overlap (step < window) the union of their pixels is staged once in
// shared memory with asynchronous copies, otherwise each thread reads its windows
// straight from global memory. The window
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

// Staged tile rows: byte (r, c) of the tile (frame pixel (x0 + c, y0 + r)) sits at
// tile[r * stride + mis(r) + c]. Word copies: mis(r) is the misalignment of that
// frame row's byte x0 (rows advance by the pitch, so it steps by pitch mod 4, mask
// 3). Bulk copies: every row has the same offset, x0 mod 16 (pmod 0, mask 15).
struct Tile {
    const uint8_t* bytes;
    int stride;
    unsigned mis0, pmod, mask;
    __device__ __forceinline__ unsigned mis(int r) const { return (mis0 + (unsigned)r * pmod) & mask; }
};

// Maximum of the 8 bytes of (lo, hi) and of acc, in two 16-bit lanes: bytes 0, 2 and
// 1, 3 of each word spread into zero-extended 16-bit lanes (byte permutes), then
// three-way 16-bit lane maxima (hardware DPX instructions since sm_90). The byte
// maximum of a row set is the larger of the result's two lanes.
__device__ __forceinline__ unsigned row_max16(unsigned lo, unsigned hi, unsigned acc)
{
    const unsigned el = __byte_perm(lo, 0u, 0x4240), ol = __byte_perm(lo, 0u, 0x4341);
    const unsigned eh = __byte_perm(hi, 0u, 0x4240), oh = __byte_perm(hi, 0u, 0x4341);
    return __vimax3_u16x2(__vimax3_u16x2(el, ol, eh), oh, acc);
}
__device__ __forceinline__ int lanes_max16(unsigned m) { return (int)max(m & 0xffffu, m >> 16); }

// Window sums of a window of width <= 8 at tile column c0, row r0: per row, the
// window's bytes become two 32-bit words (funnel shifts of three aligned loads),
// bytes past the window are masked off, and dp4a forms the row sum and the
// column-weighted row sum while 16-bit lane maxima track m.
__device__ __forceinline__ void window_sums_packed(const Tile& T, int c0, int r0, int ww, int wh, int& S, int& X,
                                                   int& Y, int& m)
{
    const unsigned mlo = ww >= 4 ? 0xffffffffu : (1u << (8 * ww)) - 1u;
    const unsigned mhi = ww >= 8 ? 0xffffffffu : ww <= 4 ? 0u : (1u << (8 * (ww - 4))) - 1u;
    const unsigned* base = reinterpret_cast<const unsigned*>(T.bytes + r0 * T.stride);
    unsigned mis = T.mis(r0);
    unsigned mx = 0;
    int s = 0, x = 0, y = 0;
    for (int i = 0; i < wh; ++i) {
        const unsigned c = (unsigned)c0 + mis;
        const unsigned* row = base + (c >> 2);
        const unsigned shift = (c & 3u) * 8u;
        const unsigned w0 = row[0], w1 = row[1], w2 = row[2];
        const unsigned lo = __funnelshift_r(w0, w1, shift) & mlo;
        const unsigned hi = __funnelshift_r(w1, w2, shift) & mhi;
        const int rs = (int)__dp4a(lo, 0x01010101u, __dp4a(hi, 0x01010101u, 0u));
        x += (int)__dp4a(lo, 0x03020100u, __dp4a(hi, 0x07060504u, 0u));
        s += rs;
        y += i * rs;
        mx = row_max16(lo, hi, mx);
        base += T.stride >> 2;
        mis = (mis + T.pmod) & T.mask;  // next row's offset
    }
    S = s;
    X = x;
    Y = y;
    m = lanes_max16(mx);
}

// Sums of the VR consecutive windows of one column (square windows of width W <= 8,
// step S, all compile-time) from a staged tile: every tile row under the column is
// read once (rows shared by overlapping windows are not re-summed); row sums, the
// column-weighted row sums and row-index-weighted row sums become prefix sums over
// the rows, so a window's S, X and Y are differences of two prefixes
// (Y = (Q_e - Q_b) - b S for the window's first row b); the maximum is a three-way
// maximum over the window's row maxima, kept as 16-bit lane pairs.
template <int W, int S, int VR>
__device__ __forceinline__ void column_window_sums(const Tile& T, int c0, int r0, int (&Sv)[VR], int (&Xv)[VR],
                                                   int (&Yv)[VR], int (&Mv)[VR])
{
    static_assert(W >= 1 && W <= 8, "packed rows hold at most 8 bytes");
    constexpr int R = (VR - 1) * S + W;  // rows under the column's windows
    constexpr unsigned mlo = W >= 4 ? 0xffffffffu : (1u << (8 * W)) - 1u;
    constexpr unsigned mhi = W >= 8 ? 0xffffffffu : W <= 4 ? 0u : (1u << (8 * (W - 4))) - 1u;
    const unsigned* base = reinterpret_cast<const unsigned*>(T.bytes + r0 * T.stride);
    unsigned mis = T.mis(r0);
    int P[R + 1], Q[R + 1], PX[R + 1];
    unsigned rm[R];
    P[0] = Q[0] = PX[0] = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const unsigned c = (unsigned)c0 + mis;
        const unsigned* row = base + r * (T.stride >> 2) + (c >> 2);
        const unsigned shift = (c & 3u) * 8u;
        const unsigned w0 = row[0], w1 = row[1];
        const unsigned lo = __funnelshift_r(w0, w1, shift) & mlo;
        const unsigned hi = W > 4 ? __funnelshift_r(w1, row[2], shift) & mhi : 0u;
        const int rs = (int)__dp4a(lo, 0x01010101u, __dp4a(hi, 0x01010101u, 0u));
        const int rx = (int)__dp4a(lo, 0x03020100u, __dp4a(hi, 0x07060504u, 0u));
        P[r + 1] = P[r] + rs;
        Q[r + 1] = Q[r] + r * rs;
        PX[r + 1] = PX[r] + rx;
        rm[r] = row_max16(lo, hi, 0u);
        mis = (mis + T.pmod) & T.mask;
    }
#pragma unroll
    for (int k = 0; k < VR; ++k) {
        const int b = k * S, e = b + W;
        Sv[k] = P[e] - P[b];
        Xv[k] = PX[e] - PX[b];
        Yv[k] = (Q[e] - Q[b]) - b * Sv[k];
        unsigned m = 0u;
#pragma unroll
        for (int i = b; i < e; i += 2) {
            unsigned next = 0u;
            if (i + 1 < e) next = rm[i + 1];
            m = __vimax3_u16x2(m, rm[i], next);
        }
        Mv[k] = lanes_max16(m);
    }
}

// Window sums of any window size, byte by byte (staged tile or frame rows).
__device__ __forceinline__ void window_sums_bytes(const uint8_t* w0, int rstride, const Tile* T, int r0, int ww,
                                                  int wh, int& S, int& X, int& Y, int& m)
{
    S = X = Y = m = 0;
    for (int i = 0; i < wh; ++i) {
        const uint8_t* row = w0 + (size_t)i * rstride + (T ? T->mis(r0 + i) : 0u);
        int rs = 0, rx = 0;
        for (int j = 0; j < ww; ++j) {
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

// Each thread owns a window column and vr consecutive windows along it; a CTA covers
// 32 x (by vr) windows of one frame, and the CTAs of all frames of the batch share
// one grid. When windows overlap (step < window) the CTA stages the union of their
// pixels (large tiles: few staging round trips per SM): with one bulk copy per row
// when the frame's base, pitch and width are multiples of 16, else with 4-byte
// copies of the aligned words holding them; otherwise threads read the frame directly.
// Four resident blocks per SM (shared memory allows four at the largest tiles): up to 64
// registers a thread, no spills.
__global__ void __launch_bounds__(256, 4) degraf_detect_kernel(const __grid_constant__ DetectBatch a)
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
    const int wy = (int)blockDim.y * a.vr;  // windows per CTA along y
    const int u0 = (t % J.tiles_x) * kBX, v0 = (t / J.tiles_x) * wy;
    const int x0 = u0 * J.step, y0 = v0 * J.step;
    const long long org = (long long)(uintptr_t)J.img + (long long)y0 * J.pitch + x0;
    const Tile T = J.bulk ? Tile{tile, a.tile_w, (unsigned)x0 & 15u, 0u, 15u}
                          : Tile{tile, a.tile_w, (unsigned)org & 3u, (unsigned)J.pitch & 3u, 3u};
    if (a.staged) {
        // tile rows past the frame are never read
        const int tw = min((kBX - 1) * J.step + a.ww, J.W - x0);
        const int th = min((wy - 1) * J.step + a.wh, J.H - y0);
        const int nthr = kBX * blockDim.y, tid = threadIdx.y * kBX + threadIdx.x;
        if (J.bulk) {
            // frame base, pitch and width multiples of 16: one bulk copy per row of
            // the 16-byte aligned span covering the tile's columns (it stays inside
            // the row), all completing on one barrier
            __shared__ __align__(8) uint64_t bar;
            if (tid == 0) mbar_init(&bar, 1);
            __syncthreads();
            const int a_lo = x0 & ~15, a_hi = (x0 + tw + 15) & ~15;
            if (tid == 0) mbar_arrive_expect_tx(&bar, (unsigned)(th * (a_hi - a_lo)));
            for (int r = tid; r < th; r += nthr)
                bulk_copy_to_smem(tile + r * a.tile_w, J.img + (long long)(y0 + r) * J.pitch + a_lo,
                                  (unsigned)(a_hi - a_lo), &bar);
            const bool ok = mbar_wait(&bar, 0, kStageWaitTries);
            if (!__syncthreads_and(ok)) {  // the copy engine stopped answering: record, drain, leave
                if (tid == 0 && a.status) atomicOr(a.status, (unsigned)DGF_DEV_STAGE_WAIT);
                mbar_wait(&bar, 0, kStageWaitTries);
                return;
            }
        } else {
            // every aligned word holding a byte of the tile (such a word lies inside
            // the frame's allocation)
            const int nwr = (tw + 3 + 3) >> 2;  // words per row, misalignment included
            for (int i = tid; i < th * nwr; i += nthr) {
                const int r = i / nwr, k = i - r * nwr;
                const int c_lo = 4 * k - (int)T.mis(r);  // tile column of the word's first byte
                if (c_lo >= tw) continue;
                cp_async4(tile + r * a.tile_w + 4 * k, J.img + (long long)(y0 + r) * J.pitch + x0 + c_lo);
            }
            cp_async_wait_all();
            __syncthreads();
        }
    }
    const int u = u0 + threadIdx.x;
    if (u >= J.nu) return;
    // common square windows: the column's four windows at once, rows shared
    if (a.staged && a.vr == 4 && a.ww == a.wh) {
        const int key = a.ww * 16 + J.step;
        if (key == 8 * 16 + 2 || key == 8 * 16 + 3 || key == 8 * 16 + 4 || key == 8 * 16 + 6 || key == 7 * 16 + 3) {
            int Sv[4], Xv[4], Yv[4], Mv[4];
            const int c0 = threadIdx.x * J.step, r0 = threadIdx.y * 4 * J.step;
            switch (key) {
                case 8 * 16 + 2: column_window_sums<8, 2, 4>(T, c0, r0, Sv, Xv, Yv, Mv); break;
                case 8 * 16 + 3: column_window_sums<8, 3, 4>(T, c0, r0, Sv, Xv, Yv, Mv); break;
                case 8 * 16 + 4: column_window_sums<8, 4, 4>(T, c0, r0, Sv, Xv, Yv, Mv); break;
                case 8 * 16 + 6: column_window_sums<8, 6, 4>(T, c0, r0, Sv, Xv, Yv, Mv); break;
                default: column_window_sums<7, 3, 4>(T, c0, r0, Sv, Xv, Yv, Mv); break;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int v = v0 + threadIdx.y * 4 + k;
                if (v < J.nv) emit(J, a.ww, a.wh, u, v, Sv[k], Xv[k], Yv[k], Mv[k]);
            }
            return;
        }
    }
    for (int k = 0; k < a.vr; ++k) {
        const int wv = threadIdx.y * a.vr + k;  // window row inside the CTA
        const int v = v0 + wv;
        if (v >= J.nv) return;
        int S, X, Y, m;
        if (a.staged && a.ww <= 8) {
            window_sums_packed(T, threadIdx.x * J.step, wv * J.step, a.ww, a.wh, S, X, Y, m);
        } else if (a.staged) {
            window_sums_bytes(tile + wv * J.step * a.tile_w + threadIdx.x * J.step, a.tile_w, &T, wv * J.step, a.ww,
                              a.wh, S, X, Y, m);
        } else {
            window_sums_bytes(J.img + (size_t)(v * J.step) * J.pitch + u * J.step, J.pitch, nullptr, 0, a.ww, a.wh, S,
                              X, Y, m);
        }
        emit(J, a.ww, a.wh, u, v, S, X, Y, m);
    }
}

// Chooses the CTA shape (32 x by threads, vr windows per thread along y; staged
// through shared memory when the windows overlap and every frame's tile fits),
// fills the CTA prefix counts and launches detection for every frame of the batch.
int launch_detect(DetectBatch& a, cudaStream_t stream)
{
    int max_step = 1;
    bool overlap = true;
    for (int f = 0; f < a.n_jobs; ++f) {
        max_step = a.jobs[f].step > max_step ? a.jobs[f].step : max_step;
        overlap = overlap && (a.jobs[f].step < a.ww || a.jobs[f].step < a.wh);
    }
    // row stride: the tile's bytes, up to 15 bytes of row offset, and room for the
    // packed path's three aligned word loads from a window's first byte; a multiple
    // of 16 for the bulk row copies
    const int tile_w = ((kBX - 1) * max_step + a.ww + 15 + 12 + 15) / 16 * 16;
    int by = 8, vr = 4;
    auto tile_h = [&]() { return (by * vr - 1) * max_step + a.wh; };
    while (tile_w * tile_h() > kSmemMax && (vr > 1 || by > 1)) {
        if (vr > 1)
            vr /= 2;
        else
            by /= 2;
    }
    a.by = by;
    a.vr = vr;
    a.staged = overlap && tile_w * tile_h() <= kSmemMax;
    a.tile_w = tile_w;  // row stride of the staged tile
    a.tile_h = tile_h();
    long long ctas = 0;
    a.status = status_word();
    for (int f = 0; f < a.n_jobs; ++f) {
        DetectJob& J = a.jobs[f];
        // rows whose 16-byte spans end at or before the row's last byte: no copy reads
        // past the frame, whatever lies beyond its last row
        J.bulk = aligned(J.img, 16) && J.pitch % 16 == 0 && J.W % 16 == 0;
        J.tiles_x = (J.nu + kBX - 1) / kBX;
        J.cta_begin = (int)ctas;
        ctas += (long long)J.tiles_x * ((J.nv + by * vr - 1) / (by * vr));
    }
    if (ctas == 0) return DGF_OK;
    if (ctas > 0x7fffffffLL) return DGF_ERR_ARG;
    degraf_detect_kernel<<<(unsigned)ctas, dim3(kBX, by), a.staged ? (size_t)a.tile_w * a.tile_h : 0, stream>>>(a);
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
