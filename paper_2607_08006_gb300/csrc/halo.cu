// GPU-resident halo exchange in a stencil code (paper Sec. 4.4, case study 1): every
// PE owns an nx x ny tile of a periodic 2-D grid (PEs in a px x py grid) and runs Jacobi
// sweeps; between sweeps its boundary rows and columns go into its four neighbours'
// halo buffers with device-initiated puts, completed by put-with-signal (Sec. 7) and
// awaited with bounded wait_until (Sec. 6.4).
//
// Symmetric objects (every PE's copy at the same offset):
//   tiles: tile[p] = tiles + p*nx*ny floats, p = 0, 1 (double buffer);
//   halos: halo[p] = halos + p*hs floats, hs = 2nx + 2ny4 (ny4 = ny rounded up to a
//          multiple of 4): [north nx][south nx][west ny4][east ny4], the neighbouring
//          values the tile's boundary reads in a sweep that reads tile[p] (every part
//          starts on a 16-byte boundary);
//   sigs:  4 uint64 [from north, from south, from west, from east], counting the halos
//          that have arrived.
// Sweep t reads tile[t&1] and halo[t&1] and writes tile[(t+1)&1]; the new boundary values
// are stored straight into the neighbours' halo[(t+1)&1] from the sweep's epilogue (no
// staging), then one release signal per neighbour.  A PE may overwrite a neighbour's
// halo[(t+1)&1] only after that neighbour has finished sweep t-1, which read it; the
// neighbour's own signal for sweep t proves that.
//
// Jacobi update, in this order: out = 0.25 * ((up + down) + (left + right)), binary32 RNE.
#include <cuda_runtime.h>

#include "internal.h"

namespace shmemg {

enum { H_N = 0, H_S = 1, H_W = 2, H_E = 3 };

struct HaloArgs {
    shmemg_device_ctx_t c;
    uint64_t tiles, halos, sigs;  // symmetric offsets
    int px, py, nx, ny;
};

// floats per halo buffer: north and south rows, west and east columns padded to a
// multiple of 4 (16-byte aligned parts, a multiple of 4 floats in all)
__host__ __device__ __forceinline__ uint64_t halo_ny4(int ny) { return ((uint64_t)ny + 3) & ~3ull; }
__host__ __device__ __forceinline__ uint64_t halo_stride(int nx, int ny) { return 2ull * nx + 2 * halo_ny4(ny); }
__host__ __device__ __forceinline__ uint64_t halo_part(int nx, int ny, int part) {
    return part == H_N ? 0 : part == H_S ? (uint64_t)nx : part == H_W ? 2ull * nx : 2ull * nx + halo_ny4(ny);
}

// Rows a thread keeps in flight on the staged path (shared-memory ring per thread).
constexpr int HALO_RING = 16;
// dynamic shared memory of the staged path: HALO_RING slots of one float4 per thread
// plus two edge float4 per warp
__host__ __device__ __forceinline__ size_t halo_smem(int threads) {
    return (size_t)HALO_RING * 16 * (threads + 2 * (threads / 32));
}

__device__ __forceinline__ void halo_cp16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void halo_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void halo_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ float jac(float up, float dn, float lf, float rt) {
    return __fmul_rn(0.25f, __fadd_rn(__fadd_rn(up, dn), __fadd_rn(lf, rt)));
}

// Rows [R0, R1) of one sweep of this PE's tile (group g: the PE's threads) from tile[p] /
// halo[p] into tile[p^1]; with `send`, the new boundary values also go to the neighbours'
// halo[p^1].  edges = false (the interior phase, rows 1 .. ny-2): the west and east
// halos are not read -- the points of columns 0 and nx-1 get a placeholder left or right
// value from the tile itself and are recomputed by halo_boundary -- so the rows can be swept
// before the neighbours' halos have arrived.
// Thread layout: float4 column c4 = rank mod W4, a contiguous run of rows per thread
// (sliding window of three rows in registers, one new float4 per row).  The grid's
// update is the same on both paths below; they differ only in where a point's left and
// right neighbours come from.
__device__ __forceinline__ void halo_sweep(const HaloArgs &a, shmemg_group g, int me, const int nb[4], int p,
                                           bool send, int R0, int R1, bool edges) {
    const shmemg_device_ctx_t &c = a.c;
    const int nx = a.nx, ny = a.ny, W4 = nx / 4;
    const uint64_t tile_elems = (uint64_t)nx * ny, halo_elems = halo_stride(nx, ny);
    const float *cur = (const float *)shmemg_d_addr(c, me, a.tiles) + (uint64_t)p * tile_elems;
    float *nxt = (float *)shmemg_d_addr(c, me, a.tiles) + (uint64_t)(p ^ 1) * tile_elems;
    const float *hal = (const float *)shmemg_d_addr(c, me, a.halos) + (uint64_t)p * halo_elems;
    const float *h_n = hal + halo_part(nx, ny, H_N), *h_s = hal + halo_part(nx, ny, H_S);
    const float *h_w = hal + halo_part(nx, ny, H_W), *h_e = hal + halo_part(nx, ny, H_E);
    // the neighbours' halo[p^1] parts this tile's boundary feeds
    auto nb_halo = [&](int dir, int part) {
        return (float *)shmemg_d_addr(c, nb[dir], a.halos) + (uint64_t)(p ^ 1) * halo_elems + halo_part(nx, ny, part);
    };
    float *to_n = nb_halo(H_N, H_S), *to_s = nb_halo(H_S, H_N);  // my top row is the north PE's south halo
    float *to_w = nb_halo(H_W, H_E), *to_e = nb_halo(H_E, H_W);
    const uint32_t T = g.size;
    const uint32_t cols = T < (uint32_t)W4 ? T : (uint32_t)W4;  // threads per row sweep
    const uint32_t nseg = T / cols;                              // row runs side by side
    if (g.rank >= cols * nseg) return;
    const uint32_t seg = g.rank / cols;
    const int r0 = R0 + (int)((uint64_t)(R1 - R0) * seg / nseg), r1 = R0 + (int)((uint64_t)(R1 - R0) * (seg + 1) / nseg);
    if (r0 >= r1) return;
    // every load bypasses L1 (ld.global.cg): neighbours and the PE's other CTAs wrote
    // these values on other SMs since this SM may last have cached them
    auto store = [&](int i, int c4, const float4 &o) {
        const int j = 4 * c4;
        *reinterpret_cast<float4 *>(nxt + (uint64_t)i * nx + j) = o;
        if (send) {  // fused device-initiated puts of the new boundary
            if (i == 0) *reinterpret_cast<float4 *>(to_n + j) = o;
            if (i == ny - 1) *reinterpret_cast<float4 *>(to_s + j) = o;
            if (c4 == 0 && edges) to_w[i] = o.x;
            if (c4 == W4 - 1 && edges) to_e[i] = o.w;
        }
    };
    auto stencil = [&](const float4 &up, const float4 &mid, const float4 &dn, float lf, float rt) {
        float4 o;
        o.x = jac(up.x, dn.x, lf, mid.y);
        o.y = jac(up.y, dn.y, mid.x, mid.z);
        o.z = jac(up.z, dn.z, mid.y, mid.w);
        o.w = jac(up.w, dn.w, mid.z, rt);
        return o;
    };
    if (cols % 32 == 0 && (blockDim.x & 31) == 0) {
        // staged warp path.  A warp covers 32 consecutive float4 columns of the same rows,
        // so a point's left and right neighbours come from the adjacent lanes by shuffle;
        // the warp's edge lanes also stage the 16-byte chunk beside them (or the chunk of
        // the west / east halo holding the row's value).  Every thread streams its column
        // through a private ring of HALO_RING shared-memory slots filled by cp.async (one
        // group per row, HALO_RING - 3 rows still in flight while a row is computed), so
        // the loads in flight do not hold registers.
        extern __shared__ __align__(16) float4 halo_ring[];
        const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5);
        const int nw = (int)(blockDim.x >> 5);
        float4 *ring = halo_ring + threadIdx.x;                       // slot k at ring[k * blockDim.x]
        float4 *edge = halo_ring + HALO_RING * blockDim.x + 2 * warp;  // slot k at edge[k * 2 * nw] (+0 left, +1 right)
        for (int cb = (int)(g.rank % cols) - lane; cb < W4; cb += (int)cols) {   // warp-uniform
            const int c4 = cb + lane;
            const bool act = c4 < W4;
            const int j = act ? 4 * c4 : 0;   // idle lanes read column 0 and store nothing
            const bool ledge = lane == 0, redge = act && (lane == 31 || c4 == W4 - 1);
            auto slot = [&](int x) { return (x - (r0 - 1)) & (HALO_RING - 1); };
            // row x (r0-1 <= x <= r1) into its slot, with the edge chunks of computed rows
            auto issue = [&](int x) {
                if (x <= r1) {
                    const int k = slot(x);
                    const float *q = x < 0 ? h_n + j : x >= ny ? h_s + j : cur + (uint64_t)x * nx + j;
                    halo_cp16(ring + k * blockDim.x, q);
                    if (x >= r0 && x < r1) {   // (edges off: rows 1 .. ny-2, so the side reads stay in the tile)
                        if (ledge)
                            halo_cp16(edge + 2 * k * nw, c4 == 0 && edges ? h_w + (x & ~3) : cur + (uint64_t)x * nx + j - 4);
                        if (redge)
                            halo_cp16(edge + 2 * k * nw + 1,
                                      c4 == W4 - 1 && edges ? h_e + (x & ~3) : cur + (uint64_t)x * nx + j + 4);
                    }
                }
                halo_commit();   // an empty group past the end keeps the count
            };
            for (int x = r0 - 1; x < r0 - 1 + HALO_RING; x++) issue(x);
            halo_wait<HALO_RING - 2>();   // rows r0 - 1 and r0 have landed
            float4 up = ring[slot(r0 - 1) * blockDim.x], mid = ring[slot(r0) * blockDim.x];
            // steady state: pointers and the slot advance by one row per step
            const bool west = ledge && c4 == 0 && edges, east = redge && c4 == W4 - 1 && edges;   // lanes on the tile's sides
            const float *nsrc = cur + (uint64_t)(r0 - 1 + HALO_RING) * nx + j;  // row i - 1 + HALO_RING
            float *dst = nxt + (uint64_t)r0 * nx + j;
            int sl = slot(r0);
#pragma unroll 4
            for (int i = r0; i < r1; i++) {
                halo_wait<HALO_RING - 3>();   // rows up to i + 1 have landed
                const int sdn = (sl + 1) & (HALO_RING - 1);
                const float4 dn = ring[sdn * blockDim.x];
                float lf = __shfl_up_sync(0xffffffffu, mid.w, 1);
                float rt = __shfl_down_sync(0xffffffffu, mid.x, 1);
                const int q = i & 3;   // a side halo's value within its 16-byte chunk
                if (ledge) {
                    const float4 e = edge[2 * sl * nw];
                    lf = !west ? e.w : q == 0 ? e.x : q == 1 ? e.y : q == 2 ? e.z : e.w;
                }
                if (redge) {
                    const float4 e = edge[2 * sl * nw + 1];
                    rt = !east ? e.x : q == 0 ? e.x : q == 1 ? e.y : q == 2 ? e.z : e.w;
                }
                const float4 o = stencil(up, mid, dn, lf, rt);
                if (act) {
                    *reinterpret_cast<float4 *>(dst) = o;
                    if (send) {  // fused device-initiated puts of the new boundary
                        if (i == 0) *reinterpret_cast<float4 *>(to_n + j) = o;
                        if (i == ny - 1) *reinterpret_cast<float4 *>(to_s + j) = o;
                        if (west) to_w[i] = o.x;
                        if (east) to_e[i] = o.w;
                    }
                }
                // row x = i - 1 + HALO_RING into row i - 1's slot (that row is in `up`)
                const int x = i - 1 + HALO_RING;
                if (x <= r1) {
                    const int si = (sl - 1) & (HALO_RING - 1);
                    halo_cp16(ring + si * blockDim.x, x < ny ? nsrc : h_s + j);
                    if (x < r1) {
                        if (ledge) halo_cp16(edge + 2 * si * nw, west ? h_w + (x & ~3) : nsrc - 4);
                        if (redge) halo_cp16(edge + 2 * si * nw + 1, east ? h_e + (x & ~3) : nsrc + 4);
                    }
                }
                halo_commit();
                nsrc += nx;
                dst += nx;
                sl = sdn;
                up = mid;
                mid = dn;
            }
            halo_wait<0>();
        }
        return;
    }
    for (int c4 = (int)(g.rank % cols); c4 < W4; c4 += (int)cols) {
        const int j = 4 * c4;
        // rows -1 and ny are the north and south halos
        auto row = [&](int i) {
            const float *q = i < 0 ? h_n + j : i >= ny ? h_s + j : cur + (uint64_t)i * nx + j;
            return __ldcg(reinterpret_cast<const float4 *>(q));
        };
        auto left = [&](int i) { return c4 == 0 && edges ? __ldcg(h_w + i) : __ldcg(cur + (uint64_t)i * nx + j - 1); };
        auto right = [&](int i) {
            return c4 == W4 - 1 && edges ? __ldcg(h_e + i) : __ldcg(cur + (uint64_t)i * nx + j + 4);
        };
        auto emit = [&](int i, const float4 &up, const float4 &mid, const float4 &dn, float lf, float rt) {
            store(i, c4, stencil(up, mid, dn, lf, rt));
        };
        float4 up = row(r0 - 1), mid = row(r0);
        int i = r0;
        for (; i + 4 <= r1; i += 4) {  // four rows' loads in flight per thread
            const float4 d0 = row(i + 1), d1 = row(i + 2), d2 = row(i + 3), d3 = row(i + 4);
            const float l0 = left(i), l1 = left(i + 1), l2 = left(i + 2), l3 = left(i + 3);
            const float q0 = right(i), q1 = right(i + 1), q2 = right(i + 2), q3 = right(i + 3);
            emit(i, up, mid, d0, l0, q0);
            emit(i + 1, mid, d0, d1, l1, q1);
            emit(i + 2, d0, d1, d2, l2, q2);
            emit(i + 3, d1, d2, d3, l3, q3);
            up = d2;
            mid = d3;
        }
        for (; i < r1; i++) {
            const float4 dn = row(i + 1);
            emit(i, up, mid, dn, left(i), right(i));
            up = mid;
            mid = dn;
        }
    }
}

// The boundary after an interior phase (ny > 2): rows 0 and ny-1 as float4 chunks, then
// columns 0 and nx-1 of rows 1 .. ny-2 as single points, with their sends.  Every load of
// a thread's items is issued before the first result is needed (four edge points per
// round), so the pass costs about two round trips.
__device__ __forceinline__ void halo_boundary(const HaloArgs &a, shmemg_group g, int me, const int nb[4], int p,
                                              bool send) {
    const shmemg_device_ctx_t &c = a.c;
    const int nx = a.nx, ny = a.ny, W4 = nx / 4;
    const uint64_t tile_elems = (uint64_t)nx * ny, halo_elems = halo_stride(nx, ny);
    const float *cur = (const float *)shmemg_d_addr(c, me, a.tiles) + (uint64_t)p * tile_elems;
    float *nxt = (float *)shmemg_d_addr(c, me, a.tiles) + (uint64_t)(p ^ 1) * tile_elems;
    const float *hal = (const float *)shmemg_d_addr(c, me, a.halos) + (uint64_t)p * halo_elems;
    const float *h_n = hal + halo_part(nx, ny, H_N), *h_s = hal + halo_part(nx, ny, H_S);
    const float *h_w = hal + halo_part(nx, ny, H_W), *h_e = hal + halo_part(nx, ny, H_E);
    auto nb_halo = [&](int dir, int part) {
        return (float *)shmemg_d_addr(c, nb[dir], a.halos) + (uint64_t)(p ^ 1) * halo_elems + halo_part(nx, ny, part);
    };
    float *to_n = nb_halo(H_N, H_S), *to_s = nb_halo(H_S, H_N), *to_w = nb_halo(H_W, H_E), *to_e = nb_halo(H_E, H_W);
    for (uint32_t q = g.rank; q < 2u * (uint32_t)W4; q += g.size) {  // a float4 chunk of row 0 or row ny-1
        const int i = q < (uint32_t)W4 ? 0 : ny - 1, c4 = (int)(q % (uint32_t)W4), j = 4 * c4;
        const float *row = cur + (uint64_t)i * nx;
        const float4 up = __ldcg(reinterpret_cast<const float4 *>(i == 0 ? h_n + j : row - nx + j));
        const float4 mid = __ldcg(reinterpret_cast<const float4 *>(row + j));
        const float4 dn = __ldcg(reinterpret_cast<const float4 *>(i == ny - 1 ? h_s + j : row + nx + j));
        const float lf = c4 == 0 ? __ldcg(h_w + i) : __ldcg(row + j - 1);
        const float rt = c4 == W4 - 1 ? __ldcg(h_e + i) : __ldcg(row + j + 4);
        float4 o;
        o.x = jac(up.x, dn.x, lf, mid.y);
        o.y = jac(up.y, dn.y, mid.x, mid.z);
        o.z = jac(up.z, dn.z, mid.y, mid.w);
        o.w = jac(up.w, dn.w, mid.z, rt);
        *reinterpret_cast<float4 *>(nxt + (uint64_t)i * nx + j) = o;
        if (send) {
            *reinterpret_cast<float4 *>((i == 0 ? to_n : to_s) + j) = o;
            if (c4 == 0) to_w[i] = o.x;
            if (c4 == W4 - 1) to_e[i] = o.w;
        }
    }
    // edge points e = 0 .. 2(ny-2)-1: row 1 + e/2, column 0 (e even) or nx-1 (e odd)
    constexpr int U = 4;
    const uint32_t nedge = 2u * (uint32_t)(ny - 2);
    for (uint32_t e0 = g.rank; e0 < nedge; e0 += U * g.size) {
        float v[U][4];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t e = e0 + (uint32_t)u * g.size;
            if (e >= nedge) continue;
            const int i = 1 + (int)(e >> 1);
            const float *row = cur + (uint64_t)i * nx;
            if ((e & 1) == 0) {
                v[u][0] = __ldcg(row - nx);
                v[u][1] = __ldcg(row + nx);
                v[u][2] = __ldcg(h_w + i);
                v[u][3] = __ldcg(row + 1);
            } else {
                v[u][0] = __ldcg(row - 1);
                v[u][1] = __ldcg(row + nx + nx - 1);
                v[u][2] = __ldcg(row + nx - 2);
                v[u][3] = __ldcg(h_e + i);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t e = e0 + (uint32_t)u * g.size;
            if (e >= nedge) continue;
            const int i = 1 + (int)(e >> 1);
            const float o = jac(v[u][0], v[u][1], v[u][2], v[u][3]);
            if ((e & 1) == 0) {
                nxt[(uint64_t)i * nx] = o;
                if (send) to_w[i] = o;
            } else {
                nxt[(uint64_t)i * nx + nx - 1] = o;
                if (send) to_e[i] = o;
            }
        }
    }
}

// The initial halos: tile[0]'s boundary into the neighbours' halo[0].
__device__ __forceinline__ void halo_prime(const HaloArgs &a, shmemg_group g, int me, const int nb[4]) {
    const shmemg_device_ctx_t &c = a.c;
    const int nx = a.nx, ny = a.ny;
    const float *t0 = (const float *)shmemg_d_addr(c, me, a.tiles);
    auto nb_halo = [&](int dir, int part) { return (float *)shmemg_d_addr(c, nb[dir], a.halos) + halo_part(nx, ny, part); };
    float *to_n = nb_halo(H_N, H_S), *to_s = nb_halo(H_S, H_N), *to_w = nb_halo(H_W, H_E), *to_e = nb_halo(H_E, H_W);
    for (uint32_t k = g.rank; k < (uint32_t)nx; k += g.size) {
        to_n[k] = __ldcg(t0 + k);
        to_s[k] = __ldcg(t0 + (uint64_t)(ny - 1) * nx + k);
    }
    for (uint32_t k = g.rank; k < (uint32_t)ny; k += g.size) {
        to_w[k] = __ldcg(t0 + (uint64_t)k * nx);
        to_e[k] = __ldcg(t0 + (uint64_t)k * nx + nx - 1);
    }
}

__device__ __forceinline__ void halo_neighbours(const HaloArgs &a, int me, int nb[4]) {
    const int x = me % a.px, y = me / a.px;
    nb[H_N] = ((y + a.py - 1) % a.py) * a.px + x;
    nb[H_S] = ((y + 1) % a.py) * a.px + x;
    nb[H_W] = y * a.px + (x + a.px - 1) % a.px;
    nb[H_E] = y * a.px + (x + 1) % a.px;
}

// signals: my data went to nb[dir]; it arrives there from the opposite direction
__device__ __forceinline__ void halo_signal(const HaloArgs &a, const int nb[4]) {
    shmemg_d_fence_gpu();
    const int from[4] = {H_S, H_N, H_E, H_W};
    for (int d = 0; d < 4; d++)
        shmemg_d_red_release_add_u64((uint64_t *)shmemg_d_addr(a.c, nb[d], a.sigs) + from[d], 1);
}

// Sweeps t0 .. t1-1 of a run of `iters`.  Persistent form (signals on): the whole run in
// one cooperative launch (t0 = 0, t1 = iters), PEs synchronised pairwise by their
// signals only.  Plain form (signals off): one launch per sweep (t1 = t0 + 1), kernel
// boundaries order the sweeps and no signal is sent or awaited; both forms run the same
// sweep code.
template <bool SPLIT>
__global__ void __launch_bounds__(512) k_halo(HaloArgs a, int t0, int t1, int iters, int signals) {
    const shmemg_device_ctx_t &c = a.c;
    const int me = shmemg_d_my_pe(c);
    const shmemg_group g = shmemg_d_group_pe(c);
    const bool leader = shmemg_d_pe_leader(c);
    __shared__ int s_stop;
    int nb[4];
    halo_neighbours(a, me, nb);
    if (threadIdx.x == 0) s_stop = 0;
    uint64_t *my_sig = (uint64_t *)shmemg_d_addr(c, me, a.sigs);
    if (signals) {
        halo_prime(a, g, me, nb);
        shmemg_d_pe_sync(c);
        if (leader) halo_signal(a, nb);
    }
    for (int t = t0; t < t1; t++) {
        const bool send = t + 1 < iters;
        // SPLIT (the persistent form, ny > 2): the interior rows first -- they read only
        // this PE's own tile, so they overlap the wait for the neighbours' halos
        if constexpr (SPLIT) halo_sweep(a, g, me, nb, t & 1, false, 1, a.ny - 1, false);
        if (signals && threadIdx.x == 0) {
            int rc = SHMEMG_SUCCESS;
            if (leader)
                for (int d = 0; d < 4 && rc == SHMEMG_SUCCESS; d++)
                    rc = shmemg_d_signal_wait_until(c, my_sig + d, SHMEMG_CMP_GE, (uint64_t)t + 1, t);
            s_stop = rc != SHMEMG_SUCCESS;
        }
        shmemg_d_pe_sync(c);
        // the leader CTA's verdict decides for the PE (in pe_mode CLUSTER the other CTAs
        // read it through DSMEM; the leader rewrites it only after the next PE barrier)
        const int stop = c.pe_mode == SHMEMG_PE_MODE_CLUSTER && c.cluster_dim > 1
                             ? shmemg_d_ld_cluster<int>(shmemg_d_cluster_addr(&s_stop, 0))
                             : s_stop;
        if (stop) break;
        // then rows 0 and ny-1 and columns 0 and nx-1 (SPLIT), or the whole tile
        if constexpr (SPLIT) halo_boundary(a, g, me, nb, t & 1, send);
        else halo_sweep(a, g, me, nb, t & 1, send, 0, a.ny, true);
        shmemg_d_pe_sync(c);
        if (signals && send && leader) halo_signal(a, nb);
    }
    if (signals) {
        // every halo meant for this PE has arrived (or the run failed): reset the
        // counters for the next run
        shmemg_d_pe_sync(c);
        if (leader)
            for (int d = 0; d < 4; d++) my_sig[d] = 0;
    }
}

// The plain form's first step: tile[0]'s boundary into the neighbours' halo[0].
__global__ void __launch_bounds__(512) k_halo_prime(HaloArgs a) {
    const int me = shmemg_d_my_pe(a.c);
    int nb[4];
    halo_neighbours(a, me, nb);
    halo_prime(a, shmemg_d_group_pe(a.c), me, nb);
}


// 512 threads per PE: one CTA of 512, or cluster_dim CTAs of 512 / cluster_dim (so a
// clustered PE spreads the same work over more SMs and every PE still fits at once)
static int halo_threads() {
    const State &S = st();
    return S.pe_mode == SHMEMG_PE_MODE_CLUSTER ? 512 / S.cluster_dim : 512;
}

// launch k_halo / k_halo_prime with the staged path's shared memory
static int halo_launch(const void *kernel, void **args, cudaStream_t s) {
    const int threads = halo_threads();
    const size_t smem = halo_smem(threads);
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return SHMEMG_ERR_UNSUPPORTED;
    }
    return launch_pe_grid(kernel, args, smem, s, threads);
}

static int halo_args(float *tiles, float *halos, uint64_t *sigs, int px, int py, int nx, int ny, int iters,
                     HaloArgs *a) {
    if (int rc = check_init()) return rc;
    State &S = st();
    if (px < 1 || py < 1 || (int64_t)px * py != S.npes || nx < 4 || nx % 4 || ny < 1 || iters < 0)
        return SHMEMG_ERR_INVALID_ARG;
    uint64_t to, ho, so;
    const uint64_t tb = 2ull * nx * ny * 4, hb = 2ull * halo_stride(nx, ny) * 4;
    if (sym_offset(tiles, tb, &to) || sym_offset(halos, hb, &ho) || sym_offset(sigs, 32, &so)) return SHMEMG_ERR_NOT_SYMMETRIC;
    if ((to | ho) & 15 || so & 7) return SHMEMG_ERR_INVALID_ARG;  // float4 rows, aligned signals
    a->c = device_ctx();
    a->tiles = to;
    a->halos = ho;
    a->sigs = so;
    a->px = px;
    a->py = py;
    a->nx = nx;
    a->ny = ny;
    return SHMEMG_SUCCESS;
}

}  // namespace shmemg

using namespace shmemg;

extern "C" uint64_t shmemg_halo_stride(int nx, int ny) { return nx < 0 || ny < 0 ? 0 : halo_stride(nx, ny); }

extern "C" int shmemg_halo_jacobi(float *tiles, float *halos, uint64_t *sigs, int px, int py, int nx, int ny,
                                  int iters, void *stream) {
    HaloArgs a;
    if (int rc = halo_args(tiles, halos, sigs, px, py, nx, ny, iters, &a)) return rc;
    if (iters == 0) return SHMEMG_SUCCESS;
    int t0 = 0, signals = 1;
    void *args[] = {(void *)&a, (void *)&t0, (void *)&iters, (void *)&iters, (void *)&signals};
    // tiles of more than two rows sweep their interior while the halos are on the way
    return halo_launch(ny > 2 ? (const void *)k_halo<true> : (const void *)k_halo<false>, args, to_stream(stream));
}

extern "C" int shmemg_halo_jacobi_plain(float *tiles, float *halos, uint64_t *sigs, int px, int py, int nx, int ny,
                                        int iters, void *stream) {
    HaloArgs a;
    if (int rc = halo_args(tiles, halos, sigs, px, py, nx, ny, iters, &a)) return rc;
    if (iters == 0) return SHMEMG_SUCCESS;
    void *pargs[] = {(void *)&a};
    if (int rc = halo_launch((const void *)k_halo_prime, pargs, to_stream(stream))) return rc;
    int t = 0, t1 = 1, signals = 0;
    void *args[] = {(void *)&a, (void *)&t, (void *)&t1, (void *)&iters, (void *)&signals};
    for (t = 0; t < iters; t++) {
        t1 = t + 1;
        if (int rc = halo_launch((const void *)k_halo<false>, args, to_stream(stream))) return rc;
    }
    return SHMEMG_SUCCESS;
}
