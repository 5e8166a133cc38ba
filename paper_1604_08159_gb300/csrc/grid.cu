// Lattice kernels: initial condition, DD reconstruction and details (Sec. 2.4,
// Eq. 6), thresholding with the adjacent zone, closure under prediction,
// stencil levels and ghost points (Sec. 2.5), and the stable multi-bucket
// compaction that turns the masks into index lists.
#include <cstdlib>

#include "kernels.h"

namespace wrc {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

template <typename T>
__global__ void k_init_vortices(T* __restrict__ L, const double* __restrict__ prm, int n, Geom g) {
    pdl_wait();
    const long long N = (long long)g.NJ * g.NJ;
    const double twopi = 2.0 * kPi;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p & g.mask), k = (int)(p >> g.L);
        const double x = -kPi + g.h * i, y = -kPi + g.h * k;
        double om = 0.0;
        for (int v = 0; v < n; ++v) {
            double dx = x - prm[v], dy = y - prm[n + v];
            dx -= twopi * floor((dx + kPi) / twopi);   // minimum image in [-pi, pi)
            dy -= twopi * floor((dy + kPi) / twopi);
            const double s2 = prm[3 * n + v] * prm[3 * n + v];
            om += prm[2 * n + v] / (kPi * s2) * exp(-(dx * dx + dy * dy) / s2);
        }
        L[p] = (T)om;
    }
    pdl_trigger();
}

// With rows (see launch_scatter): the pair q of rows 2q, 2q+1 within margin
// rows of a grid point is flagged (rows[q]) and, by the thread that flags it
// first, appended to the list rows[h + 1 ..] (count at rows[h]; any order).
__device__ __forceinline__ void flag_pair(int* rows, int h, int q) {
    if (*(volatile int*)(rows + q)) return;
    if (atomicExch(rows + q, 1) == 0) rows[h + 1 + atomicAdd(rows + h, 1)] = q;
}

template <typename T>
__global__ void k_scatter(const uint32_t* __restrict__ meta, const T* __restrict__ vals, long long n,
                          T* __restrict__ L, const int* __restrict__ dn, int* __restrict__ rows, int margin,
                          int lg, int mask) {
    pdl_wait();
    n = eff_n(dn, n);
    const int h = (mask + 1) >> 1;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const uint32_t p = meta_pos(meta[a]);
        L[p] = vals[a];
        if (rows) {
            // one lane per distinct row among the warp's points flags its pairs
            const int k = (int)(p >> lg);
            const unsigned same = __match_any_sync(__activemask(), k);
            if ((int)(threadIdx.x & 31) == __ffs(same) - 1) {
                for (int d = -margin; d <= margin; d += 2) flag_pair(rows, h, ((k + d) & mask) >> 1);
                flag_pair(rows, h, ((k + margin) & mask) >> 1);
            }
        }
    }
    pdl_trigger();
}

// Coarse-to-fine inverse transform for one level: every non-active level-j
// point gets its DD prediction (its detail is zero, Eq. 6), in two passes.
// Pass 1: the points odd in one direction only (one 1-D prediction each),
// the first n^2/4 indices odd rows and even columns, the next n^2/4 even rows
// and odd columns (n = NJ / 2^(J-j) points per row at this level).
template <typename T>
__global__ void k_recon_level_1d(T* __restrict__ L, const uint8_t* __restrict__ act, int j, Geom g) {
    pdl_wait();
    const int sh = g.J - j;
    const int lh = g.L - sh - 1;             // log2(n / 2)
    const int q = 1 << (2 * lh);             // n^2 / 4
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * q; t += gridDim.x * blockDim.x) {
        const int u = t < q ? t : t - q;
        const int r = u >> lh, c = u & ((1 << lh) - 1);
        const int k = (t < q ? 2 * r + 1 : 2 * r) << sh;
        const int i = (t < q ? 2 * c : 2 * c + 1) << sh;
        const long long p = ((long long)k << g.L) + i;
        if (!act[p]) L[p] = predict<T>(L, i, k, j, g);
    }
    pdl_trigger();
}

// Pass 2: the points odd in both directions.  Their prediction is the y
// prediction over the x predictions of rows k -+ s, k -+ 3s, .. (2P rows) at
// column i, and those x predictions are exactly the values pass 1 stored at
// the points (i, k -+ s), (i, k -+ 3s), .. unless these are active (same
// operands, same rounded operations): only the rows of active neighbours are
// predicted again.  Bit-identical to the tensor-product predictor, with one 1-D
// prediction per point instead of five for most points.
template <typename T, int P>
__global__ void k_recon_level_2d(T* __restrict__ L, const uint8_t* __restrict__ act, int j, Geom g) {
    pdl_wait();
    const int sh = g.J - j;
    const int s = 1 << sh, m = g.mask;
    const int lh = g.L - sh - 1;
    const int q = 1 << (2 * lh);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < q; t += gridDim.x * blockDim.x) {
        const int r = t >> lh, c = t & ((1 << lh) - 1);
        const int k = (2 * r + 1) << sh, i = (2 * c + 1) << sh;
        const long long p = ((long long)k << g.L) + i;
        if (act[p]) continue;
        if constexpr (P == 2) {
            const int ks[4] = {(k - s) & m, (k + s) & m, (k - 3 * s) & m, (k + 3 * s) & m};
            T rv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const long long pe = ((long long)ks[e] << g.L) + i;
                if (!act[pe]) {
                    rv[e] = L[pe];
                } else {
                    const T* row = L + ((size_t)ks[e] << g.L);
                    rv[e] = dd4<T>(row[(i - s) & m], row[(i + s) & m], row[(i - 3 * s) & m], row[(i + 3 * s) & m]);
                }
            }
            L[p] = dd4<T>(rv[0], rv[1], rv[2], rv[3]);
        } else {
            // rows k -+ (2e + 1) s: the x prediction stored there by pass 1, or
            // computed again where that point is active
            T lo[P], hi[P];
#pragma unroll
            for (int e = 0; e < P; ++e) {
                const int o = (2 * e + 1) * s;
                const int kl = (k - o) & m, kh = (k + o) & m;
                const long long pl = ((long long)kl << g.L) + i, ph = ((long long)kh << g.L) + i;
                lo[e] = act[pl] ? predict_line<T, P, false>(L, i, kl, s, true, g) : L[pl];
                hi[e] = act[ph] ? predict_line<T, P, false>(L, i, kh, s, true, g) : L[ph];
            }
            L[p] = ddp<T, P>(lo, hi);
        }
    }
    pdl_trigger();
}

// Regions of a tile's reconstruction along one axis: level J is the tile
// [t0, t0 + ts); level j - 1 covers level j widened by the predictor's reach
// (2P - 1) 2^(J-j) on each side, rounded outward to the level-(j-1) lattice.
// lo[j]: first coordinate (fine units; may lie outside [0, NJ): periodic);
// n[j]: number of level-j lattice points.  The sizes depend on t0 only
// modulo the coarsest spacing 2^J.
constexpr int kReconLevels = 11;   // J <= 10
struct TileAxis {
    int lo[kReconLevels];
    int n[kReconLevels];
};
struct ReconTiles {
    int ts, tiles_x, bytes, pmax;
    int off[kReconLevels];     // level j's values in shared memory (elements of T)
    int aoff[kReconLevels];    // level j's grid flags (bytes from the start)
    int pitch[kReconLevels];   // row length of both; value rows: pitch + 2 (2P - 1)
};
constexpr int kReconPitchMax = 64;   // a level's region holds at most 64^2 points

__host__ __device__ inline void tile_axis(int t0, int ts, int J, int P, TileAxis& a) {
    int lo = t0, hi = t0 + ts - 1;
    a.lo[J] = lo;
    a.n[J] = ts;
    for (int j = J; j >= 1; --j) {
        const int r = (2 * P - 1) << (J - j);
        const int sh = J - j + 1;   // log2 of the level-(j-1) spacing
        lo = ((lo - r) >> sh) << sh;
        hi = ((hi + r + (1 << sh) - 1) >> sh) << sh;
        a.lo[j - 1] = lo;
        a.n[j - 1] = ((hi - lo) >> sh) + 1;
    }
}

// Tile size and shared-memory layout for the tiled reconstruction (the
// largest tile of at most 64^2 whose arrays fit kReconSmemMax); false when
// none does (the level-by-level kernels are used then).
constexpr int kReconSmemMax = 160 * 1024;
bool recon_tiles_layout(const Geom& g, size_t es, ReconTiles& lay) {
    if (g.J >= kReconLevels) return false;
    const int E = 2 * g.P - 1;
    // tile edge: 64 up to 1024^2 (on GB300 at 1024^2, J = 5: 64 before 32, 16
    // and the level-by-level kernels); beyond, the level-by-level kernels,
    // whose passes then have parallelism enough (4096^2, J = 7: 0.22 ms
    // against 0.33 ms tiled); WRC_RECON_TILE sets the edge (0: level by level)
    int cap = g.NJ <= 1024 ? 64 : 0;
    if (const char* v = std::getenv("WRC_RECON_TILE")) cap = std::atoi(v);
    if (cap < 8) return false;   // 0: the level-by-level kernels
    for (int ts = g.NJ < cap ? g.NJ : cap; ts >= 8 && ts <= g.NJ; ts /= 2) {
        int nmax[kReconLevels] = {0};
        const int per = 1 << g.J;
        for (int t0 = 0; t0 < (per > ts ? per : ts); t0 += ts) {
            TileAxis a;
            tile_axis(t0, ts, g.J, g.P, a);
            for (int j = 0; j <= g.J; ++j) nmax[j] = a.n[j] > nmax[j] ? a.n[j] : nmax[j];
        }
        long long off = 0;
        int pmax = 0;
        for (int j = 0; j <= g.J; ++j) {
            lay.off[j] = (int)off;
            lay.pitch[j] = nmax[j];
            off += (long long)(nmax[j] + 2 * E) * nmax[j];
            pmax = nmax[j] > pmax ? nmax[j] : pmax;
        }
        long long b = off * (long long)es;
        for (int j = 0; j <= g.J; ++j) {
            lay.aoff[j] = (int)b;
            b += (long long)nmax[j] * nmax[j];
        }
        if (pmax <= kReconPitchMax && b <= kReconSmemMax) {
            lay.pmax = pmax;
            lay.ts = ts;
            lay.tiles_x = g.NJ / ts;
            lay.bytes = (int)b;
            return true;
        }
    }
    return false;
}

// Entry t = u + v n of a loop over rows n wide, t advancing by kThreads,
// without a division per step.
struct RowWalk {
    int u, v, du, dv, n;
    __device__ __forceinline__ RowWalk(int t, int n_) : n(n_) {
        u = t % n;
        v = t / n;
        du = kThreads % n;
        dv = kThreads / n;
    }
    __device__ __forceinline__ void next() {
        u += du;
        v += dv;
        if (u >= n) {
            u -= n;
            ++v;
        }
    }
};

// The whole coarse-to-fine inverse transform in one launch, one tile of the
// finest lattice per block.  A block reconstructs the values of every level
// over its tile widened, level by level, by the predictor's reach (points
// of the level-j lattice within (2P - 1) 2^(J-j) fine cells of the region
// of level j + 1), in shared memory: levels are not synchronised across
// blocks; each block recomputes the coarse values its tile depends on.
// At level j, phase 1 copies the points of level j - 1 and makes the 1-D
// predictions: of the points odd in x only (also in 2P - 1 extra rows above
// and below the region, for phase 2) and of those odd in y only; phase 2
// predicts the points odd in both directions from the x predictions of
// phase 1 (the tensor product, y over x, as predict does); phase 3 puts the
// values of grid points in place of their predictions and stores the
// non-grid points of the tile.  The operations and their order are those of
// the level-by-level kernels, so L is bit-identical.  Only non-grid points
// are written, each by the block whose tile holds it; grid points are only
// read.
// FP64 issue is a bound (a warp instruction costs the same whatever the
// number of active lanes), so each loop enumerates only its own kind of
// point: every lane of a warp makes a prediction of the same form, from
// operands at base - q d and base + (1 + q) d (d = 1 along x, the row pitch
// along y).  Loads are issued ahead of their use: each level's grid values
// into registers before its predictions (used in phase 3), the next level's
// grid flags during this level's predictions.
template <typename T, int P, int PMAX>
__global__ void __launch_bounds__(kThreads) k_recon_tiles(T* __restrict__ L, const uint8_t* __restrict__ act, Geom g,
                                                          ReconTiles lay) {
    extern __shared__ __align__(16) unsigned char recon_smem[];
    T* sm = reinterpret_cast<T*>(recon_smem);
    constexpr int E = 2 * P - 1;   // extra rows of x predictions on each side
    constexpr int kPre = (PMAX * PMAX + kThreads - 1) / kThreads;   // entries of a region per thread
    const int ts = lay.ts, m = g.mask;
    const int x0 = (int)(blockIdx.x % lay.tiles_x) * ts, y0 = (int)(blockIdx.x / lay.tiles_x) * ts;
    TileAxis ax, ay;
    tile_axis(x0, ts, g.J, P, ax);
    tile_axis(y0, ts, g.J, P, ay);
    // grid flags of the level-j points of level j's region (entries
    // threadIdx.x + t kThreads): loaded into fv, then stored to shared memory
    uint8_t fv[kPre];
    auto load_flags = [&](int j) {
        const int sh = g.J - j, nx = ax.n[j], ny = ay.n[j];
        RowWalk w(threadIdx.x, nx);
#pragma unroll
        for (int t = 0; t < kPre; ++t) {
            fv[t] = 0;
            if (w.v >= ny) break;
            const int i = ax.lo[j] + (w.u << sh), k = ay.lo[j] + (w.v << sh);
            if (((i >> sh) | (k >> sh)) & 1) fv[t] = act[((size_t)(k & m) << g.L) + (i & m)];
            w.next();
        }
    };
    auto store_flags = [&](int j) {
        const int nx = ax.n[j], ny = ay.n[j], pitch = lay.pitch[j];
        uint8_t* F = recon_smem + lay.aoff[j];
        RowWalk w(threadIdx.x, nx);
#pragma unroll
        for (int t = 0; t < kPre; ++t) {
            if (w.v >= ny) break;
            F[w.v * pitch + w.u] = fv[t];
            w.next();
        }
    };
    pdl_wait();
    load_flags(1);
    {
        // level 0: every point is a grid point (and is never written)
        T* A = sm + lay.off[0];
        const int pitch = lay.pitch[0], nx = ax.n[0], ny = ay.n[0], sh = g.J;
        for (int e = threadIdx.x; e < nx * ny; e += kThreads) {
            const int c = e % nx, r = e / nx;
            const int i = (ax.lo[0] + (c << sh)) & m, k = (ay.lo[0] + (r << sh)) & m;
            A[(r + E) * pitch + c] = L[((size_t)k << g.L) + i];
        }
    }
    store_flags(1);
    __syncthreads();
    for (int j = 1; j <= g.J; ++j) {
        const int sh = g.J - j;
        const T* C = sm + lay.off[j - 1];
        const int cp = lay.pitch[j - 1], cx0 = ax.lo[j - 1], cy0 = ay.lo[j - 1];
        T* A = sm + lay.off[j];
        const uint8_t* F = recon_smem + lay.aoff[j];
        const int pitch = lay.pitch[j], nx = ax.n[j], ny = ay.n[j], lx = ax.lo[j], ly = ay.lo[j];
        // this thread's grid values of phase 3 (entries threadIdx.x + t kThreads)
        T pv[kPre];
        {
            RowWalk w(threadIdx.x, nx);
#pragma unroll
            for (int t = 0; t < kPre; ++t) {
                pv[t] = T(0);
                if (w.v >= ny) break;
                if (F[w.v * pitch + w.u])
                    pv[t] = L[((size_t)((ly + (w.v << sh)) & m) << g.L) + ((lx + (w.u << sh)) & m)];
                w.next();
            }
        }
        if (j < g.J) load_flags(j + 1);
        // first odd and even columns, even rows (all), odd rows (the region's)
        const int co0 = ((lx >> sh) & 1) ? 0 : 1, ce0 = 1 - co0;
        const int nxo = (nx - co0 + 1) >> 1, nxe = (nx - ce0 + 1) >> 1;
        const int re0 = ((ly >> sh) - E) & 1, nre = (ny + 2 * E - re0 + 1) >> 1;
        const int ro0 = E + (((ly >> sh) & 1) ? 0 : 1), nro = (ny - (ro0 - E) + 1) >> 1;
        // row rr of A holds fine row ly + (rr - E) s; its level-(j-1) row in C
        // is (rr - E + (ly - cy0) / s) / 2 + E, its column c is (c + (lx - cx0) / s) / 2
        const int dr = (ly - cy0) >> sh, dc = (lx - cx0) >> sh;
        if (nxo > 0) {   // odd in x only: along the row, from level j - 1
            RowWalk w(threadIdx.x, nxo);
#pragma unroll 4
            for (int t = threadIdx.x; t < nxo * nre; t += kThreads) {
                const int c = co0 + 2 * w.u, rr = re0 + 2 * w.v;
                const int b = (((rr - E + dr) >> 1) + E) * cp + ((c - 1 + dc) >> 1);
                T lo[P], hi[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    lo[q] = C[b - q];
                    hi[q] = C[b + 1 + q];
                }
                A[rr * pitch + c] = ddp<T, P>(lo, hi);
                w.next();
            }
        }
        if (nxe > 0) {   // odd in y only: along the column
            RowWalk w(threadIdx.x, nxe);
#pragma unroll 4
            for (int t = threadIdx.x; t < nxe * nro; t += kThreads) {
                const int c = ce0 + 2 * w.u, rr = ro0 + 2 * w.v;
                const int b = (((rr - 1 - E + dr) >> 1) + E) * cp + ((c + dc) >> 1);
                T lo[P], hi[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    lo[q] = C[b - q * cp];
                    hi[q] = C[b + (1 + q) * cp];
                }
                A[rr * pitch + c] = ddp<T, P>(lo, hi);
                w.next();
            }
            RowWalk wc(threadIdx.x, nxe);
#pragma unroll 4
            for (int t = threadIdx.x; t < nxe * nre; t += kThreads) {   // points of level j - 1
                const int c = ce0 + 2 * wc.u, rr = re0 + 2 * wc.v;
                A[rr * pitch + c] = C[(((rr - E + dr) >> 1) + E) * cp + ((c + dc) >> 1)];
                wc.next();
            }
        }
        __syncthreads();
        if (nxo > 0) {   // odd in both: y over the x predictions
            RowWalk w(threadIdx.x, nxo);
#pragma unroll 4
            for (int t = threadIdx.x; t < nxo * nro; t += kThreads) {
                const int c = co0 + 2 * w.u, r = ro0 + 2 * w.v;
                T lo[P], hi[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    lo[q] = A[(r - (2 * q + 1)) * pitch + c];
                    hi[q] = A[(r + (2 * q + 1)) * pitch + c];
                }
                A[r * pitch + c] = ddp<T, P>(lo, hi);
                w.next();
            }
        }
        __syncthreads();
        {
            RowWalk w(threadIdx.x, nx);
#pragma unroll
            for (int t = 0; t < kPre; ++t) {
                if (w.v >= ny) break;
                const int i = lx + (w.u << sh), k = ly + (w.v << sh);
                if (((i >> sh) | (k >> sh)) & 1) {
                    T* a = A + (w.v + E) * pitch + w.u;
                    if (F[w.v * pitch + w.u]) *a = pv[t];
                    else if (i >= x0 && i < x0 + ts && k >= y0 && k < y0 + ts)
                        L[((size_t)(k & m) << g.L) + (i & m)] = *a;
                }
                w.next();
            }
        }
        if (j < g.J) store_flags(j + 1);
        __syncthreads();
    }
    pdl_trigger();
}

// Values at the new points of a rebuilt grid (in `nxt`, not in `act`) for
// one level: the DD prediction from the current grid's values (Eq. 6, detail
// zero), tensor form for points odd in both directions.  Every predictor
// point of a new point is in the closed new grid: a current point (value in
// L) or a coarser new point (written by an earlier level's launch).  The
// other non-current points are not written.
template <typename T>
__global__ void k_recon_new(T* __restrict__ L, const uint8_t* __restrict__ act, const uint8_t* __restrict__ nxt,
                            int j, Geom g) {
    pdl_wait();
    const long long cnt = level_count(j, g);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * blockDim.x) {
        int i, k;
        level_point(t, j, g, i, k);
        const long long p = ((long long)k << g.L) + i;
        if (nxt[p] && !act[p]) L[p] = predict<T>(L, i, k, j, g);
    }
    pdl_trigger();
}

// k_recon_new for the finest level J, 16 consecutive lattice points per
// thread: the new-grid and grid flags read as 16-byte vectors (neither is
// written here), the chunks without a new point skipped.
template <typename T>
__global__ void k_recon_new_fine(T* __restrict__ L, const uint8_t* __restrict__ act,
                                 const uint8_t* __restrict__ nxt, Geom g) {
    pdl_wait();
    const long long N16 = (long long)g.NJ * g.NJ / 16;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N16;
         c += (long long)gridDim.x * blockDim.x) {
        const uint4 a = reinterpret_cast<const uint4*>(act)[c], x = reinterpret_cast<const uint4*>(nxt)[c];
        const uint32_t nw[4] = {x.x & ~a.x, x.y & ~a.y, x.z & ~a.z, x.w & ~a.w};   // flags are 0 or 1
        if (!(nw[0] | nw[1] | nw[2] | nw[3])) continue;
        for (int u = 0; u < 16; ++u) {
            if (!((nw[u >> 2] >> (8 * (u & 3))) & 0xffu)) continue;
            const long long p = 16 * c + u;
            const int i = (int)(p & g.mask), k = (int)(p >> g.L);
            if ((i | k) & 1) L[p] = predict<T>(L, i, k, g.J, g);
        }
    }
    pdl_trigger();
}

// Details d = u - Pred(u) at the active points (meta == nullptr: every lattice
// point), significance |d| >= eps (level 0 always significant), and the
// adjacent zone of every significant point of level j >= 1: the points of
// level j and j+1 within 2^(J-j) fine cells in x and y.  All writes to the
// masks store the value 1, so concurrent writers agree.
template <typename T>
__global__ void k_details_adj(const uint32_t* __restrict__ meta, long long n, const T* __restrict__ L,
                              double eps, T* __restrict__ det, uint8_t* __restrict__ sig,
                              uint8_t* __restrict__ nxt, Geom g, const int* __restrict__ dn) {
    pdl_wait();
    n = eff_n(dn, n);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const long long p = meta ? (long long)meta_pos(meta[a]) : a;
        const int i = (int)(p & g.mask), k = (int)(p >> g.L);
        const int lev = level_of(i, k, g.J);
        T d = T(0);
        bool s = true;
        if (lev > 0) {
            d = rsub(L[p], predict<T>(L, i, k, lev, g));
            s = fabs((double)d) >= eps;
        }
        if (det) det[a] = d;
        if (!s) continue;
        sig[p] = 1;
        nxt[p] = 1;
        if (lev == 0) continue;
        const int r = 1 << (g.J - lev);
        const int step = lev < g.J ? (r >> 1) : r;
        for (int dk = -r; dk <= r; dk += step) {
            const int qk = (k + dk) & g.mask;
            for (int di = -r; di <= r; di += step) {
                const int qi = (i + di) & g.mask;
                const int lq = level_of(qi, qk, g.J);
                if (lq == lev || lq == lev + 1) nxt[((long long)qk << g.L) + qi] = 1;
            }
        }
    }
    pdl_trigger();
}

// Visit the DD predictor points (order 2 g.P) of level-j point (i, k): the
// odd multiples of the level's spacing up to (2P - 1) along its odd
// direction(s), or their 2P x 2P tensor product.
template <typename F>
__device__ __forceinline__ void for_predictor_points(int i, int k, int j, const Geom& g, F&& f) {
    const int sh = g.J - j;
    const int s = 1 << sh;
    const bool oi = (i >> sh) & 1, ok = (k >> sh) & 1;
    const int np = 2 * g.P;
    if (oi && !ok) {
        for (int q = 0; q < np; ++q) f((i + (2 * q + 1 - np) * s) & g.mask, k);
    } else if (!oi && ok) {
        for (int q = 0; q < np; ++q) f(i, (k + (2 * q + 1 - np) * s) & g.mask);
    } else {
        for (int b = 0; b < np; ++b)
            for (int q = 0; q < np; ++q) f((i + (2 * q + 1 - np) * s) & g.mask, (k + (2 * b + 1 - np) * s) & g.mask);
    }
}

// Closure under prediction for one level (finest first): every marked level-j
// point marks its predictor points, except where `excl` is set.
__global__ void k_closure_level(uint8_t* __restrict__ mask, const uint8_t* __restrict__ excl, int j, Geom g) {
    pdl_wait();
    const long long cnt = level_count(j, g);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * blockDim.x) {
        int i, k;
        level_point(t, j, g, i, k);
        if (!mask[((long long)k << g.L) + i]) continue;
        for_predictor_points(i, k, j, g, [&](int qi, int qk) {
            const long long q = ((long long)qk << g.L) + qi;
            if (!excl || !excl[q]) mask[q] = 1;
        });
    }
    pdl_trigger();
}

// The closure pass of the finest level J, 16 consecutive lattice points per
// thread: their level-J marks (odd row or odd column) are read as separate
// bytes, all in flight, and never the coarser points' bytes, which the pass
// writes.
__global__ void k_closure_fine(uint8_t* __restrict__ mask, const uint8_t* __restrict__ excl, Geom g) {
    pdl_wait();
    const long long N16 = (long long)g.NJ * g.NJ / 16;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N16;
         c += (long long)gridDim.x * blockDim.x) {
        uint8_t b[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const long long p = 16 * c + u;
            const int i = (int)(p & g.mask), k = (int)(p >> g.L);
            b[u] = ((i | k) & 1) ? mask[p] : 0;
        }
        for (int u = 0; u < 16; ++u) {
            if (!b[u]) continue;
            const long long p = 16 * c + u;
            const int i = (int)(p & g.mask), k = (int)(p >> g.L);
            for_predictor_points(i, k, g.J, g, [&](int qi, int qk) {
                const long long q = ((long long)qk << g.L) + qi;
                if (!excl || !excl[q]) mask[q] = 1;
            });
        }
    }
    pdl_trigger();
}

// Stencil levels and ghost marks (each thread reads the flags of 16
// consecutive lattice points at once, NJ^2 being a multiple of 64, and
// skips them when none is a grid point).  For an active point P of level l the
// stencil level along x is the largest j in [l, J] with an active point at
// P +- h_j e_x (l if none); the stencils read P +- r h_{j*}, r = 1 .. R
// (R = 2 for 2P = 4, max(2P - 2, P) in general), and the non-active ones
// among them are ghosts.  Same along y.
__global__ void k_stencil_ghost(const uint8_t* __restrict__ act, uint8_t* __restrict__ gho,
                                uint8_t* __restrict__ JJ, Geom g) {
    pdl_wait();
    const long long N16 = (long long)g.NJ * g.NJ / 16;
    const int R = dd_reach(g.P);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N16;
         c += (long long)gridDim.x * blockDim.x) {
        const uint4 v = reinterpret_cast<const uint4*>(act)[c];
        if (!(v.x | v.y | v.z | v.w)) continue;
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
        for (int u = 0; u < 16; ++u) {
            if (!((wv[u >> 2] >> (8 * (u & 3))) & 0xffu)) continue;
            const long long p = 16 * c + u;
            const int i = (int)(p & g.mask), k = (int)(p >> g.L);
            const int lev = level_of(i, k, g.J);
            const uint8_t* row = act + ((long long)k << g.L);
            int jx = lev, jy = lev;
            for (int j = g.J; j > lev; --j) {
                const int s = 1 << (g.J - j);
                if (row[(i + s) & g.mask] || row[(i - s) & g.mask]) {
                    jx = j;
                    break;
                }
            }
            for (int j = g.J; j > lev; --j) {
                const int s = 1 << (g.J - j);
                if (act[((long long)((k + s) & g.mask) << g.L) + i] ||
                    act[((long long)((k - s) & g.mask) << g.L) + i]) {
                    jy = j;
                    break;
                }
            }
            JJ[p] = (uint8_t)(jx | (jy << 4));
            const int sx = 1 << (g.J - jx), sy = 1 << (g.J - jy);
            for (int o = -R; o <= R; ++o) {
                if (o == 0) continue;
                const long long qx = ((long long)k << g.L) + ((i + o * sx) & g.mask);
                if (!act[qx]) gho[qx] = 1;
                const long long qy = ((long long)((k + o * sy) & g.mask) << g.L) + i;
                if (!act[qy]) gho[qy] = 1;
            }
        }
    }
    pdl_trigger();
}

__global__ void k_validate_grid(const uint8_t* __restrict__ act, int* __restrict__ flag, Geom g) {
    pdl_wait();
    const long long N = (long long)g.NJ * g.NJ;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p & g.mask), k = (int)(p >> g.L);
        const int lev = level_of(i, k, g.J);
        if (lev == 0) {
            if (!act[p]) atomicOr(flag, 1);
            continue;
        }
        if (!act[p]) continue;
        bool ok = true;
        for_predictor_points(i, k, lev, g, [&](int qi, int qk) {
            if (!act[((long long)qk << g.L) + qi]) ok = false;
        });
        if (!ok) atomicOr(flag, 2);
    }
    pdl_trigger();
}

// ---- stable multi-bucket compaction -----------------------------------------
// key(p) = 0 for an active point, j for a ghost of level j, -1 otherwise; the
// output list holds bucket 0, then bucket 1, ..., each in lattice order.

// Keys of the 16 consecutive lattice points p0 .. p0 + 15 of one thread
// (p0 a multiple of 16; NJ^2 is a multiple of 64): the active and ghost masks
// read as one 16-byte vector each.
__device__ __forceinline__ void keys16(const uint8_t* __restrict__ act, const uint8_t* __restrict__ gho, long long p0,
                                       long long N, const Geom& g, int (&key)[16]) {
    if (p0 >= N) {
#pragma unroll
        for (int u = 0; u < 16; ++u) key[u] = -1;
        return;
    }
    const uint4 va = *reinterpret_cast<const uint4*>(act + p0);
    const uint4 vh = *reinterpret_cast<const uint4*>(gho + p0);
    const uint32_t wa[4] = {va.x, va.y, va.z, va.w}, wh[4] = {vh.x, vh.y, vh.z, vh.w};
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const uint32_t ab = (wa[u >> 2] >> (8 * (u & 3))) & 0xffu;
        const uint32_t hb = (wh[u >> 2] >> (8 * (u & 3))) & 0xffu;
        const long long p = p0 + u;
        key[u] = ab ? 0 : (hb ? level_of((int)(p & g.mask), (int)(p >> g.L), g.J) : -1);
    }
}

// Counts per key of one tile of kTile = 16 kThreads points (thread t: points
// 16 t .. 16 t + 15 of the tile), key-major into blk_counts[key][block].
__global__ void __launch_bounds__(kThreads) k_compact_count(const uint8_t* __restrict__ act,
                                                            const uint8_t* __restrict__ gho, Geom g, int nkeys,
                                                            int* __restrict__ blk_counts) {
    pdl_wait();
    __shared__ int s_w[kThreads / 32][kMaxKeys];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long N = (long long)g.NJ * g.NJ;
    int key[16];
    keys16(act, gho, (long long)blockIdx.x * kTile + 16LL * threadIdx.x, N, g, key);
#pragma unroll
    for (int kk = 0; kk < kMaxKeys; ++kk) {
        if (kk >= nkeys) break;
        int c = 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) c += key[u] == kk;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) s_w[wid][kk] = c;
    }
    __syncthreads();
    if (threadIdx.x < nkeys) {
        int c = 0;
        for (int w = 0; w < kThreads / 32; ++w) c += s_w[w][threadIdx.x];
        // key-major: the scan reads each key's counts contiguously
        blk_counts[(long long)threadIdx.x * gridDim.x + blockIdx.x] = c;
    }
    pdl_trigger();
}

// Exclusive scan of v over a block of 1024 threads; *total receives the sum.
__device__ int block_excl_scan_1024(int v, int& total) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    const int excl = x - v + (wid > 0 ? ws[wid - 1] : 0);
    total = ws[31];
    __syncthreads();
    return excl;
}

// Offsets of each block's bucket entries (key-major arrays, [key][block]):
// one block of 1024 threads, thread t taking a contiguous chunk of blocks;
// the chunk's counts are read once into registers (up to kScanChunk blocks,
// more in further rounds), the bucket bases are added when written.
constexpr int kScanChunk = 4;

__global__ void __launch_bounds__(1024) k_compact_scan(const int* __restrict__ blk_counts, int nblk, int nkeys,
                                                       int* __restrict__ blk_off, int* __restrict__ counts) {
    pdl_wait();
    __shared__ int s_tot[kMaxKeys];
    const int chunk = (nblk + 1023) / 1024;
    const int b0 = threadIdx.x * chunk;
    const int b1 = min(b0 + chunk, nblk);
    int base = 0;   // bucket base: the totals of the keys before kk
    for (int kk = 0; kk < nkeys; ++kk) {
        const int* cnt = blk_counts + (long long)kk * nblk;
        int* off = blk_off + (long long)kk * nblk;
        int c[kScanChunk];
        int sum = 0;
        for (int b = b0; b < b1; b += kScanChunk) {
#pragma unroll
            for (int u = 0; u < kScanChunk; ++u) c[u] = b + u < b1 ? cnt[b + u] : 0;
#pragma unroll
            for (int u = 0; u < kScanChunk; ++u) sum += c[u];
        }
        int total;
        const int excl = block_excl_scan_1024(sum, total);
        int run = base + excl;
        if (b1 - b0 <= kScanChunk) {   // the counts are still in c
#pragma unroll
            for (int u = 0; u < kScanChunk; ++u)
                if (b0 + u < b1) {
                    off[b0 + u] = run;
                    run += c[u];
                }
        } else {
            for (int b = b0; b < b1; ++b) {
                off[b] = run;
                run += cnt[b];
            }
        }
        if (threadIdx.x == 0) s_tot[kk] = total;
        base += total;
    }
    __syncthreads();
    if (threadIdx.x < nkeys) counts[threadIdx.x] = s_tot[threadIdx.x];
    pdl_trigger();
}

// Stable scatter of one tile: thread t's entries of key k go after those of
// the threads before it (an exclusive scan over the block per key) and the
// block's base offset, in lattice order.
// A tile without an entry (its counts from k_compact_count all zero, as in
// most tiles of a large lattice) returns at once.
__global__ void __launch_bounds__(kThreads) k_compact_scatter(const uint8_t* __restrict__ act,
                                                              const uint8_t* __restrict__ gho, Geom g, int nkeys,
                                                              const int* __restrict__ blk_off,
                                                              const int* __restrict__ blk_counts,
                                                              int* __restrict__ list) {
    pdl_wait();
    __shared__ int s_base[kMaxKeys];
    __shared__ int s_w[kThreads / 32][kMaxKeys];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int mine = threadIdx.x < nkeys ? blk_counts[(long long)threadIdx.x * gridDim.x + blockIdx.x] : 0;
    if (!__syncthreads_or(mine)) {
        pdl_trigger();
        return;
    }
    if (threadIdx.x < nkeys) s_base[threadIdx.x] = blk_off[(long long)threadIdx.x * gridDim.x + blockIdx.x];
    const long long N = (long long)g.NJ * g.NJ;
    const long long p0 = (long long)blockIdx.x * kTile + 16LL * threadIdx.x;
    int key[16];
    keys16(act, gho, p0, N, g, key);
    int cnt[kMaxKeys], incl[kMaxKeys];
#pragma unroll
    for (int kk = 0; kk < kMaxKeys; ++kk) {
        int c = 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) c += key[u] == kk;
        cnt[kk] = c;
        int x = c;   // inclusive scan over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        incl[kk] = x;
        if (lane == 31 && kk < nkeys) s_w[wid][kk] = x;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kMaxKeys; ++kk) {
        if (kk >= nkeys || cnt[kk] == 0) continue;
        int off = s_base[kk] + incl[kk] - cnt[kk];
        for (int w = 0; w < wid; ++w) off += s_w[w][kk];
#pragma unroll
        for (int u = 0; u < 16; ++u)
            if (key[u] == kk) list[off++] = (int)(p0 + u);
    }
    pdl_trigger();
}

template <typename T>
__global__ void k_finalize(const int* __restrict__ list, long long n, const uint8_t* __restrict__ JJ,
                           const T* __restrict__ L, uint32_t* __restrict__ meta, T* __restrict__ omega,
                           const int* __restrict__ dn) {
    pdl_wait();
    n = eff_n(dn, n);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const int p = list[a];
        const int jj = JJ[p];
        meta[a] = pack_meta(p, jj & 15, jj >> 4);
        omega[a] = L[p];
    }
    pdl_trigger();
}

// Ghost values of one level from coarser active/ghost values (coarse to fine).
template <typename T>
__global__ void k_ghost_fill(T* __restrict__ F, const int* __restrict__ glist, long long n, int j, Geom g,
                             const int* __restrict__ kstop, int jstep) {
    pdl_wait();
    if (kstop && jstep >= *kstop) return;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const int p = glist[a];
        F[p] = predict<T>(F, p & g.mask, p >> g.L, j, g);
    }
    pdl_trigger();
}

__global__ void k_level_counts(const uint32_t* __restrict__ meta, long long n, unsigned long long* counts, Geom g) {
    pdl_wait();
    __shared__ unsigned int sc[16];
    if (threadIdx.x < 16) sc[threadIdx.x] = 0;
    __syncthreads();
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const int p = meta_pos(meta[a]);
        atomicAdd(&sc[level_of(p & g.mask, p >> g.L, g.J)], 1u);
    }
    __syncthreads();
    if (threadIdx.x <= g.J && sc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)sc[threadIdx.x]);
    pdl_trigger();
}

__global__ void k_meta_to_mask(const uint32_t* __restrict__ meta, long long n, uint8_t* __restrict__ mask) {
    pdl_wait();
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        mask[meta_pos(meta[a])] = 1;
    pdl_trigger();
}

__global__ void k_list_to_mask(const int* __restrict__ list, long long n, uint8_t* __restrict__ mask) {
    pdl_wait();
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        mask[list[a]] = 1;
    pdl_trigger();
}

__global__ void k_meta_unpack(const uint32_t* __restrict__ meta, long long n, int* idx, uint8_t* jx, uint8_t* jy) {
    pdl_wait();
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const uint32_t m = meta[a];
        if (idx) idx[a] = meta_pos(m);
        if (jx) jx[a] = (uint8_t)meta_jx(m);
        if (jy) jy[a] = (uint8_t)meta_jy(m);
    }
    pdl_trigger();
}

// Index of every grid point in the combined numbering: active points
// 0..n_a-1, then the ghosts n_a.. in list order.
__global__ void k_lat2idx(const int* __restrict__ list, long long n, int* __restrict__ lat2idx,
                          const int* __restrict__ dcounts, int nkeys) {
    pdl_wait();
    if (dcounts) {
        n = 0;
        for (int q = 0; q < nkeys; ++q) n += dcounts[q];
    }
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        lat2idx[list[t]] = (int)t;
    pdl_trigger();
}

// ---- interpolation rows of all ghosts in one launch ----------------------
// The ghosts are numbered in list order, coarser levels first, and a ghost's
// row depends only on rows of coarser ghosts.  Each warp takes the next
// ghost number from a counter (in increasing order), waits until the rows of
// its ghost predictors are published, builds its row and publishes it (a
// release store of its ready flag after the row's writes).  The smallest
// unfinished number depends only on smaller numbers, which were all taken
// by running warps and are finished, so the waits always end, whatever the
// number of resident warps.  Each wait is also bounded by limit_ns (bit 1 of
// *err when it runs out; the next Krylov step then stops and reports it).

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The warp's next ghost number (lane 0 takes it from the counter *next).
__device__ __forceinline__ long long next_ghost(int* next, long long ng, int lane) {
    int t = 0;
    if (lane == 0) t = atomicAdd(next, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    return t < ng ? (long long)t : ng;
}

__device__ __forceinline__ void wait_ready(const int* flag, int* err, unsigned long long limit_ns) {
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v) return;
        if (*(volatile int*)err & 2) return;   // another wait ran out
        if (it == 0) {
            t0 = globaltimer_ns();
        } else if (globaltimer_ns() - t0 > limit_ns) {
            atomicOr(err, 2);
            return;
        }
    }
}

// The row of ghost gi is complete (every lane's writes ordered before lane
// 0's release store of the flag).
__device__ __forceinline__ void publish_ready(int* flag, int lane) {
    __syncwarp();
    if (lane == 0) asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(flag), "r"(1) : "memory");
    __syncwarp();
}

// Interpolation rows of the ghosts: the value of a ghost is the DD
// prediction from its predictor points, which are active points or ghosts
// of coarser levels (whose rows are published first); substituting gives the ghost
// as a weighted sum of active values.  The weights are products of the DD4
// weights (-1, 9, 9, -1)/16, exact binary fractions, and repeated points are
// merged, so the rows are exact.  A row longer than rmax sets *overflow.
// One warp per ghost at a time.  Lane q < 16 takes predictor q (order: a fastest, then
// b; 4 predictors for a 1-D prediction, 16 for the tensor product), looks up
// its grid index and, for a ghost, its row length; the rows (up to
// kRowStage entries each) are then staged in shared memory with all loads in
// flight, and merged in predictor order by all lanes at once -- a row's
// entries are distinct, so each entry either adds to one existing entry or
// is appended, new entries in row order.  The entries, their order and their
// sums are those of merging the terms one by one.  An entry finds its place
// through a per-warp hash table in shared memory (key: the active point,
// value: its slot in the row; open addressing, linear probing), instead of
// a scan of the row built so far.  The predictor weights are products of
// (-1, 9, 9, -1)/16, from a constant table.
constexpr int kRowWarps = 4;   // warps (ghosts in flight) per block
constexpr int kRowStage = 32;  // staged entries per predictor row (longer rows read the rest directly)
constexpr int kRowHash = 128;  // hash slots per warp (at least twice the row capacity)
__constant__ double c_dd4w[4] = {-0.0625, 0.5625, 0.5625, -0.0625};

__device__ __forceinline__ int row_hash(int key) { return (int)(((unsigned)key * 2654435761u) >> 25); }

__global__ void __launch_bounds__(32 * kRowWarps)
k_ghost_rows(const int* __restrict__ list, const int* __restrict__ lat2idx, int* __restrict__ row_len,
             int* __restrict__ row_idx, double* __restrict__ row_w, int rmax, Geom g, int* __restrict__ overflow,
             const int* __restrict__ dcounts, int nkeys, int* __restrict__ ready, int* __restrict__ err,
             unsigned long long limit_ns, int stall) {
    pdl_wait();
    constexpr int kCap = 64;
    static_assert(kRowHash >= 2 * kCap && (kRowHash & (kRowHash - 1)) == 0 && kRowHash == 128, "row_hash gives 7 bits");
    __shared__ int s_idx[kRowWarps][kCap];
    __shared__ double s_wt[kRowWarps][kCap];
    __shared__ int s_pi[kRowWarps][16][kRowStage];
    __shared__ double s_pw[kRowWarps][16][kRowStage];
    __shared__ int s_hkey[kRowWarps][kRowHash];   // -1: empty
    __shared__ int s_hval[kRowWarps][kRowHash];   // slot of the key in the row
    __shared__ int s_hpos[kRowWarps][kCap];       // hash slot of row entry e (for clearing)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* idx = s_idx[wid];
    double* wt = s_wt[wid];
    int* hkey = s_hkey[wid];
    int* hval = s_hval[wid];
    int* hpos = s_hpos[wid];
    for (int h = lane; h < kRowHash; h += 32) hkey[h] = -1;
    __syncwarp();
    long long n_act = dcounts[0], n_tot = 0;   // key 0: active points, key l: ghosts of level l
    for (int q = 0; q < nkeys; ++q) n_tot += dcounts[q];
    const long long ng = n_tot - n_act;
    const int cap = rmax < kCap ? rmax : kCap;
    for (;;) {
        if (ng <= 0) break;   // no ghosts: the counter is not touched
        const long long gi = next_ghost(ready + ng, ng, lane);   // ghost number, in list order
        if (gi >= ng) break;
        if (stall && gi == 0 && lane == 0) wait_ready(ready + gi, err, limit_ns);   // test switch: runs out
        const int p = list[n_act + gi];
        const int i = p & g.mask, k = p >> g.L;
        const int sh = g.J - level_of(i, k, g.J);
        const int s = 1 << sh;
        const bool oi = (i >> sh) & 1, ok = (k >> sh) & 1;
        const bool two_d = oi == ok;                    // odd-odd: tensor product of two 1-D predictions
        const int np = two_d ? 16 : 4;
        // lane q < np: predictor q = (a, b) = (q % 4, q / 4)
        int my_id = -1, my_rl = 0;
        if (lane < np) {
            const int a = lane & 3, b = lane >> 2;
            const int off_a = (2 * a - 3) * s, off_b = (2 * b - 3) * s;   // -3s, -s, s, 3s
            int qi = i, qk = k;
            if (two_d) {
                qi = (i + off_a) & g.mask;
                qk = (k + off_b) & g.mask;
            } else if (oi) {
                qi = (i + off_a) & g.mask;
            } else {
                qk = (k + off_a) & g.mask;
            }
            my_id = lat2idx[((long long)qk << g.L) + qi];
            if (my_id >= n_act && my_id < n_tot) {   // a coarser ghost: its row once published
                wait_ready(ready + (my_id - n_act), err, limit_ns);
                my_rl = row_len[my_id - n_act];
            } else {
                my_rl = 1;
            }
        }
        __syncwarp();
        // stage the predictor rows (their loads all in flight)
        for (int q = 0; q < np; ++q) {
            const int id = __shfl_sync(0xffffffffu, my_id, q);
            const int rl = __shfl_sync(0xffffffffu, my_rl, q);
            if (id >= n_act && id < n_tot && lane < rl && lane < kRowStage) {
                const long long r = id - n_act;
                s_pi[wid][q][lane] = row_idx[r * rmax + lane];
                s_pw[wid][q][lane] = row_w[r * rmax + lane];
            }
        }
        __syncwarp();
        int len = 0;
        bool over = false;
        for (int q = 0; q < np; ++q) {
            const int id = __shfl_sync(0xffffffffu, my_id, q);
            const int rl0 = __shfl_sync(0xffffffffu, my_rl, q);
            // weight of predictor q: a product of two DD4 weights (exact), or one
            const double w = two_d ? c_dd4w[q & 3] * c_dd4w[q >> 2] : c_dd4w[q];
            if (id < 0 || id >= n_tot) {                 // not a grid point: record, do not read
                over = true;
                continue;
            }
            const bool ghost = id >= n_act;
            const int rl = ghost ? rl0 : 1;
            const long long r = id - n_act;
            for (int e0 = 0; e0 < rl; e0 += 32) {
                const int e = e0 + lane;
                const bool has = e < rl;
                int my = 0;
                double mw = 0.0;
                if (has) {
                    if (!ghost) {
                        my = id;
                        mw = w;
                    } else if (e < kRowStage) {
                        my = s_pi[wid][q][e];
                        mw = w * s_pw[wid][q][e];
                    } else {
                        my = row_idx[r * rmax + e];
                        mw = w * row_w[r * rmax + e];
                    }
                }
                int pos = -1;
                if (has)
                    for (int h = row_hash(my);; h = (h + 1) & (kRowHash - 1)) {
                        const int key = hkey[h];
                        if (key == my) {
                            pos = hval[h];
                            break;
                        }
                        if (key < 0) break;
                    }
                if (pos >= 0) wt[pos] += mw;
                const unsigned fresh = __ballot_sync(0xffffffffu, has && pos < 0);
                if (has && pos < 0) {
                    const int slot = len + __popc(fresh & ((1u << lane) - 1u));
                    if (slot < cap) {
                        idx[slot] = my;
                        wt[slot] = mw;
                        // distinct keys in one round: a claimed slot is another key's
                        for (int h = row_hash(my);; h = (h + 1) & (kRowHash - 1))
                            if (atomicCAS(&hkey[h], -1, my) == -1) {
                                hval[h] = slot;
                                hpos[slot] = h;
                                break;
                            }
                    }
                }
                const int nf = __popc(fresh);
                if (len + nf > cap) over = true;
                len = len + nf < cap ? len + nf : cap;
                __syncwarp();
            }
        }
        for (int e = lane; e < len; e += 32) {
            row_idx[gi * rmax + e] = idx[e];
            row_w[gi * rmax + e] = wt[e];
            hkey[hpos[e]] = -1;   // empty the table for the next ghost
        }
        if (lane == 0) {
            row_len[gi] = len;
            if (over) atomicOr(overflow, 4);
        }
        publish_ready(ready + gi, lane);
    }
    pdl_trigger();
}

// Interpolation rows of the ghosts for DD orders 2P > 4: as k_ghost_rows
// (same order of work, waits and publication; same merge in predictor order, same per-warp hash table),
// with 2P or (2P)^2 predictors, their weights dd_pred(P, .) 2^-shift (products
// of two for the tensor product), rows of up to dd_row_max(P) entries, and the
// predictors' rows read from global memory (no staging).
template <int P>
__global__ void __launch_bounds__(32 * kRowWarps)
k_ghost_rows_wide(const int* __restrict__ list, const int* __restrict__ lat2idx, int* __restrict__ row_len,
                  int* __restrict__ row_idx, double* __restrict__ row_w, int rmax, Geom g, int* __restrict__ overflow,
                  const int* __restrict__ dcounts, int nkeys, int* __restrict__ ready, int* __restrict__ err,
                  unsigned long long limit_ns, int stall) {
    pdl_wait();
    constexpr int kCapW = dd_row_max(P);
    constexpr int kHashW = 2 * kCapW;
    constexpr int kHashBits = P == 3 ? 8 : 9;
    static_assert((1 << kHashBits) == kHashW, "hash table of 2 kCapW slots");
    constexpr int NP1 = 2 * P;
    __shared__ int s_idx[kRowWarps][kCapW];
    __shared__ double s_wt[kRowWarps][kCapW];
    __shared__ int s_hkey[kRowWarps][kHashW];   // -1: empty
    __shared__ int s_hval[kRowWarps][kHashW];
    __shared__ int s_hpos[kRowWarps][kCapW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* idx = s_idx[wid];
    double* wt = s_wt[wid];
    int* hkey = s_hkey[wid];
    int* hval = s_hval[wid];
    int* hpos = s_hpos[wid];
    for (int h = lane; h < kHashW; h += 32) hkey[h] = -1;
    __syncwarp();
    long long n_act = dcounts[0], n_tot = 0;
    for (int q = 0; q < nkeys; ++q) n_tot += dcounts[q];
    const long long ng = n_tot - n_act;
    const int cap = rmax < kCapW ? rmax : kCapW;
    if (ng <= 0) {   // no ghosts: the counter is not touched
        pdl_trigger();
        return;
    }
    const double scale = 1.0 / (double)(1 << dd_shift(P));
    auto w1 = [&](int a) {   // weight of the a-th predictor along one axis
        const int o = 2 * a + 1 - NP1;
        return dd_pred(P, ((o < 0 ? -o : o) - 1) >> 1) * scale;
    };
    auto hash = [](int key) { return (int)(((unsigned)key * 2654435761u) >> (32 - kHashBits)); };
    for (;;) {
        const long long gi = next_ghost(ready + ng, ng, lane);
        if (gi >= ng) break;
        if (stall && gi == 0 && lane == 0) wait_ready(ready + gi, err, limit_ns);   // test switch: runs out
        const int p = list[n_act + gi];
        const int i = p & g.mask, k = p >> g.L;
        const int sh = g.J - level_of(i, k, g.J);
        const int s = 1 << sh;
        const bool oi = (i >> sh) & 1, ok = (k >> sh) & 1;
        const bool two_d = oi == ok;
        const int np = two_d ? NP1 * NP1 : NP1;
        int len = 0;
        bool over = false;
        for (int q0 = 0; q0 < np; q0 += 32) {
            int my_id = -1, my_rl = 0;
            const int qm = q0 + lane;
            if (qm < np) {
                const int a = two_d ? qm % NP1 : qm, b = two_d ? qm / NP1 : 0;
                int qi = i, qk = k;
                if (two_d) {
                    qi = (i + (2 * a + 1 - NP1) * s) & g.mask;
                    qk = (k + (2 * b + 1 - NP1) * s) & g.mask;
                } else if (oi) {
                    qi = (i + (2 * a + 1 - NP1) * s) & g.mask;
                } else {
                    qk = (k + (2 * a + 1 - NP1) * s) & g.mask;
                }
                my_id = lat2idx[((long long)qk << g.L) + qi];
                if (my_id >= n_act && my_id < n_tot) {   // a coarser ghost: its row once published
                    wait_ready(ready + (my_id - n_act), err, limit_ns);
                    my_rl = row_len[my_id - n_act];
                } else {
                    my_rl = 1;
                }
            }
            __syncwarp();
            const int nq = np - q0 < 32 ? np - q0 : 32;
            for (int qq = 0; qq < nq; ++qq) {
                const int qg = q0 + qq;
                const int id = __shfl_sync(0xffffffffu, my_id, qq);
                const int rl0 = __shfl_sync(0xffffffffu, my_rl, qq);
                const double w = two_d ? w1(qg % NP1) * w1(qg / NP1) : w1(qg);
                if (id < 0 || id >= n_tot) {   // not a grid point: record, do not read
                    over = true;
                    continue;
                }
                const bool ghost = id >= n_act;
                const int rl = ghost ? rl0 : 1;
                const long long r = id - n_act;
                for (int e0 = 0; e0 < rl; e0 += 32) {
                    const int e = e0 + lane;
                    const bool has = e < rl;
                    int my = 0;
                    double mw = 0.0;
                    if (has) {
                        if (!ghost) {
                            my = id;
                            mw = w;
                        } else {
                            my = row_idx[r * rmax + e];
                            mw = w * row_w[r * rmax + e];
                        }
                    }
                    int pos = -1;
                    if (has)
                        for (int h = hash(my);; h = (h + 1) & (kHashW - 1)) {
                            const int key = hkey[h];
                            if (key == my) {
                                pos = hval[h];
                                break;
                            }
                            if (key < 0) break;
                        }
                    if (pos >= 0) wt[pos] += mw;
                    const unsigned fresh = __ballot_sync(0xffffffffu, has && pos < 0);
                    if (has && pos < 0) {
                        const int slot = len + __popc(fresh & ((1u << lane) - 1u));
                        if (slot < cap) {
                            idx[slot] = my;
                            wt[slot] = mw;
                            for (int h = hash(my);; h = (h + 1) & (kHashW - 1))
                                if (atomicCAS(&hkey[h], -1, my) == -1) {
                                    hval[h] = slot;
                                    hpos[slot] = h;
                                    break;
                                }
                        }
                    }
                    const int nf = __popc(fresh);
                    if (len + nf > cap) over = true;
                    len = len + nf < cap ? len + nf : cap;
                    __syncwarp();
                }
            }
        }
        for (int e = lane; e < len; e += 32) {
            row_idx[gi * rmax + e] = idx[e];
            row_w[gi * rmax + e] = wt[e];
            hkey[hpos[e]] = -1;
        }
        if (lane == 0) {
            row_len[gi] = len;
            if (over) atomicOr(overflow, 4);
        }
        publish_ready(ready + gi, lane);
    }
    pdl_trigger();
}

// The ghost-row kernel of the DD order of g.
using RowsKernel = void (*)(const int*, const int*, int*, int*, double*, int, Geom, int*, const int*, int, int*, int*,
                            unsigned long long, int);
RowsKernel rows_kernel(const Geom& g) {
    if (g.P == 3) return k_ghost_rows_wide<3>;
    if (g.P == 4) return k_ghost_rows_wide<4>;
    return k_ghost_rows;
}

}  // namespace

template <typename T>
void launch_init_vortices(T* L, const double* params, int n, const Geom& g, cudaStream_t s) {
    { launch_pdl(k_init_vortices<T>, blocks_for((long long)g.NJ * g.NJ), kThreads, 0, s, L, params, n, g); note_launch(); }
}
template <typename T>
void launch_scatter(const uint32_t* meta, const T* vals, long long n, T* L, cudaStream_t s, const int* dn,
                    int* rows, int margin, const Geom* g) {
    const int lg = g ? g->L : 0, mask = g ? g->mask : 0;
    if (!g) rows = nullptr;
    if (n > 0) { launch_pdl(k_scatter<T>, blocks_for(n), kThreads, 0, s, meta, vals, n, L, dn, rows, margin, lg, mask); note_launch(); }
}
template <typename T>
void launch_recon_level(T* L, const uint8_t* act, int j, const Geom& g, cudaStream_t s) {
    const long long q = level_count(j, g) / 3;   // n^2 / 4
    { launch_pdl(k_recon_level_1d<T>, blocks_for(2 * q), kThreads, 0, s, L, act, j, g); note_launch(); }
    if (g.P == 3) launch_pdl(k_recon_level_2d<T, 3>, blocks_for(q), kThreads, 0, s, L, act, j, g);
    else if (g.P == 4) launch_pdl(k_recon_level_2d<T, 4>, blocks_for(q), kThreads, 0, s, L, act, j, g);
    else launch_pdl(k_recon_level_2d<T, 2>, blocks_for(q), kThreads, 0, s, L, act, j, g);
    note_launch();
}
template <typename T>
void launch_recon_new(T* L, const uint8_t* act, const uint8_t* nxt, const Geom& g, cudaStream_t s) {
    for (int j = 1; j < g.J; ++j) {
        launch_pdl(k_recon_new<T>, blocks_for(level_count(j, g)), kThreads, 0, s, L, act, nxt, j, g);
        note_launch();
    }
    launch_pdl(k_recon_new_fine<T>, blocks_for((long long)g.NJ * g.NJ / 16), kThreads, 0, s, L, act, nxt, g);
    note_launch();
}
template <typename T>
void launch_reconstruct(T* L, const uint8_t* act, const Geom& g, cudaStream_t s) {
    ReconTiles lay;
    if (recon_tiles_layout(g, sizeof(T), lay)) {
        auto k = lay.pmax <= 32
                     ? (g.P == 3 ? k_recon_tiles<T, 3, 32> : (g.P == 4 ? k_recon_tiles<T, 4, 32> : k_recon_tiles<T, 2, 32>))
                     : (g.P == 3 ? k_recon_tiles<T, 3, 64> : (g.P == 4 ? k_recon_tiles<T, 4, 64> : k_recon_tiles<T, 2, 64>));
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.bytes);
        launch_pdl(k, lay.tiles_x * lay.tiles_x, kThreads, lay.bytes, s, L, act, g, lay);
        note_launch();
        return;
    }
    for (int j = 1; j <= g.J; ++j) launch_recon_level<T>(L, act, j, g, s);
}
template <typename T>
void launch_details_adj(const uint32_t* meta, long long n, const T* L, double eps, T* det, uint8_t* sig,
                        uint8_t* nxt, const Geom& g, cudaStream_t s, const int* dn) {
    if (n > 0) { launch_pdl(k_details_adj<T>, blocks_for(n), kThreads, 0, s, meta, n, L, eps, det, sig, nxt, g, dn); note_launch(); }
}
void launch_closure_level(uint8_t* mask, const uint8_t* excl, int j, const Geom& g, cudaStream_t s) {
    if (j == g.J)
        launch_pdl(k_closure_fine, blocks_for((long long)g.NJ * g.NJ / 16), kThreads, 0, s, mask, excl, g);
    else
        launch_pdl(k_closure_level, blocks_for(level_count(j, g)), kThreads, 0, s, mask, excl, j, g);
    note_launch();
}
void launch_stencil_ghost(const uint8_t* act, uint8_t* gho, uint8_t* JJ, const Geom& g, cudaStream_t s) {
    { launch_pdl(k_stencil_ghost, blocks_for((long long)g.NJ * g.NJ / 16), kThreads, 0, s, act, gho, JJ, g); note_launch(); }
}
void launch_validate_grid(const uint8_t* act, int* flag, const Geom& g, cudaStream_t s) {
    { launch_pdl(k_validate_grid, blocks_for((long long)g.NJ * g.NJ), kThreads, 0, s, act, flag, g); note_launch(); }
}
void launch_compact(const uint8_t* act, const uint8_t* gho, const Geom& g, int nkeys, int* blk_counts,
                    int* blk_off, int* counts, int* list, cudaStream_t s) {
    const long long N = (long long)g.NJ * g.NJ;
    const int nblk = (int)((N + kTile - 1) / kTile);
    { launch_pdl(k_compact_count, nblk, kThreads, 0, s, act, gho, g, nkeys, blk_counts); note_launch(); }
    { launch_pdl(k_compact_scan, 1, 1024, 0, s, blk_counts, nblk, nkeys, blk_off, counts); note_launch(); }
    { launch_pdl(k_compact_scatter, nblk, kThreads, 0, s, act, gho, g, nkeys, (const int*)blk_off,
                 (const int*)blk_counts, list); note_launch(); }
}
template <typename T>
void launch_finalize(const int* list, long long n, const uint8_t* JJ, const T* L, uint32_t* meta, T* omega,
                     cudaStream_t s, const int* dn) {
    if (n > 0) { launch_pdl(k_finalize<T>, blocks_for(n), kThreads, 0, s, list, n, JJ, L, meta, omega, dn); note_launch(); }
}
template <typename T>
void launch_ghost_fill(T* F, const int* glist, long long n, int j, const Geom& g, const int* kstop, int jstep,
                       cudaStream_t s) {
    if (n > 0) { launch_pdl(k_ghost_fill<T>, blocks_for(n), kThreads, 0, s, F, glist, n, j, g, kstop, jstep); note_launch(); }
}
void launch_level_counts(const uint32_t* meta, long long n, unsigned long long* counts, const Geom& g,
                         cudaStream_t s) {
    if (n > 0) { launch_pdl(k_level_counts, blocks_for(n), kThreads, 0, s, meta, n, counts, g); note_launch(); }
}
void launch_meta_to_mask(const uint32_t* meta, long long n, uint8_t* mask, cudaStream_t s) {
    if (n > 0) { launch_pdl(k_meta_to_mask, blocks_for(n), kThreads, 0, s, meta, n, mask); note_launch(); }
}
void launch_list_to_mask(const int* list, long long n, uint8_t* mask, cudaStream_t s) {
    if (n > 0) { launch_pdl(k_list_to_mask, blocks_for(n), kThreads, 0, s, list, n, mask); note_launch(); }
}
void launch_ghost_rows(const int* list, int J, int* lat2idx, int* row_len, int* row_idx, double* row_w, int rmax,
                       const Geom& g, int* overflow, int* ready, int* err, unsigned long long limit_ns,
                       cudaStream_t s, const int* dcounts, long long cap_a, long long cap_g) {
    // sizes on the device, grids over the capacities (capturable)
    { launch_pdl(k_lat2idx, blocks_for(cap_a + cap_g), kThreads, 0, s, list, cap_a + cap_g, lat2idx, dcounts, J + 1); note_launch(); }
    if (!ready || cap_g <= 0) return;   // no ghost capacity: no rows
    cudaMemsetAsync(ready, 0, sizeof(int) * (size_t)(cap_g + 1), s);   // flags and the ghost counter
    // test switch: the first ghost's warp waits for a flag nothing sets
    const char* sv = std::getenv("WRC_TEST_GHOST_STALL");
    const int stall = sv && std::atoi(sv) != 0;
    launch_pdl(rows_kernel(g), blocks_for(cap_g, kRowWarps), 32 * kRowWarps, 0, s, list, (const int*)lat2idx, row_len,
               row_idx, row_w, rmax, g, overflow, dcounts, J + 1, ready, err, limit_ns, stall);
    note_launch();
}
void launch_meta_unpack(const uint32_t* meta, long long n, int* idx, uint8_t* jx, uint8_t* jy, cudaStream_t s) {
    if (n > 0) { launch_pdl(k_meta_unpack, blocks_for(n), kThreads, 0, s, meta, n, idx, jx, jy); note_launch(); }
}

#define WRC_INST(T)                                                                                       \
    template void launch_init_vortices<T>(T*, const double*, int, const Geom&, cudaStream_t);             \
    template void launch_scatter<T>(const uint32_t*, const T*, long long, T*, cudaStream_t, const int*,     \
                                    int*, int, const Geom*);                                              \
    template void launch_reconstruct<T>(T*, const uint8_t*, const Geom&, cudaStream_t);                   \
    template void launch_recon_new<T>(T*, const uint8_t*, const uint8_t*, const Geom&, cudaStream_t);     \
    template void launch_details_adj<T>(const uint32_t*, long long, const T*, double, T*, uint8_t*,       \
                                        uint8_t*, const Geom&, cudaStream_t, const int*);                 \
    template void launch_finalize<T>(const int*, long long, const uint8_t*, const T*, uint32_t*, T*,      \
                                     cudaStream_t, const int*);                                           \
    template void launch_ghost_fill<T>(T*, const int*, long long, int, const Geom&, const int*, int,      \
                                       cudaStream_t);
WRC_INST(double)
WRC_INST(float)
#undef WRC_INST

}  // namespace wrc
