// GPU-resident halo exchange in a stencil code (paper Sec. 4.4, case study 1): every
// PE owns an nx x ny tile of a periodic 2-D grid (PEs in a px x py grid) and runs Jacobi
// sweeps; between sweeps its boundary rows and columns go into its four neighbours'
// halo buffers with device-initiated puts, completed by put-with-signal (Sec. 7) and
// awaited with bounded wait_until (Sec. 6.4).
//
// Symmetric objects (every PE's copy at the same offset):
//   tiles: tile[p] = tiles + p*nx*ny floats, p = 0, 1 (double buffer);
//   halos: halo[p] = halos + p*hs floats, hs = 2nx + 2ny rounded up to a multiple of 4:
//          [north nx][south nx][west ny][east ny], the neighbouring values the tile's
//          boundary reads in a sweep that reads tile[p];
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

// floats per halo buffer (16-byte multiple, so both parities keep float4 alignment)
__host__ __device__ __forceinline__ uint64_t halo_stride(int nx, int ny) {
    return (2ull * nx + 2ull * ny + 3) & ~3ull;
}

__device__ __forceinline__ float jac(float up, float dn, float lf, float rt) {
    return __fmul_rn(0.25f, __fadd_rn(__fadd_rn(up, dn), __fadd_rn(lf, rt)));
}

// One sweep of this PE's tile (group g: the PE's threads) from tile[p] / halo[p] into
// tile[p^1]; with `send`, the new boundary values also go to the neighbours' halo[p^1].
// Thread layout: float4 column c4 = rank mod W4, a contiguous run of rows per thread
// (sliding window of three rows in registers, one new float4 per row).
__device__ __forceinline__ void halo_sweep(const HaloArgs &a, shmemg_group g, int me, const int nb[4], int p,
                                           bool send) {
    const shmemg_device_ctx_t &c = a.c;
    const int nx = a.nx, ny = a.ny, W4 = nx / 4;
    const uint64_t tile_elems = (uint64_t)nx * ny, halo_elems = halo_stride(nx, ny);
    const float *cur = (const float *)shmemg_d_addr(c, me, a.tiles) + (uint64_t)p * tile_elems;
    float *nxt = (float *)shmemg_d_addr(c, me, a.tiles) + (uint64_t)(p ^ 1) * tile_elems;
    const float *hal = (const float *)shmemg_d_addr(c, me, a.halos) + (uint64_t)p * halo_elems;
    const float *h_n = hal, *h_s = hal + nx, *h_w = hal + 2 * nx, *h_e = hal + 2 * nx + ny;
    // the neighbours' halo[p^1] parts this tile's boundary feeds
    auto nb_halo = [&](int dir, int part) {
        return (float *)shmemg_d_addr(c, nb[dir], a.halos) + (uint64_t)(p ^ 1) * halo_elems +
               (part == H_N ? 0 : part == H_S ? nx : part == H_W ? 2 * nx : 2 * nx + ny);
    };
    float *to_n = nb_halo(H_N, H_S), *to_s = nb_halo(H_S, H_N);  // my top row is the north PE's south halo
    float *to_w = nb_halo(H_W, H_E), *to_e = nb_halo(H_E, H_W);
    const uint32_t T = g.size;
    const uint32_t cols = T < (uint32_t)W4 ? T : (uint32_t)W4;  // threads per row sweep
    const uint32_t nseg = T / cols;                              // row runs side by side
    if (g.rank >= cols * nseg) return;
    const uint32_t seg = g.rank / cols;
    const int r0 = (int)((uint64_t)ny * seg / nseg), r1 = (int)((uint64_t)ny * (seg + 1) / nseg);
    if (r0 >= r1) return;
    for (int c4 = (int)(g.rank % cols); c4 < W4; c4 += (int)cols) {
        const int j = 4 * c4;
        // rows -1 and ny are the north and south halos; every load bypasses L1
        // (ld.global.cg): neighbours and the PE's other CTAs wrote these values on other
        // SMs since this SM may last have cached them
        auto row = [&](int i) {
            const float *q = i < 0 ? h_n + j : i >= ny ? h_s + j : cur + (uint64_t)i * nx + j;
            return __ldcg(reinterpret_cast<const float4 *>(q));
        };
        auto left = [&](int i) { return c4 == 0 ? __ldcg(h_w + i) : __ldcg(cur + (uint64_t)i * nx + j - 1); };
        auto right = [&](int i) { return c4 == W4 - 1 ? __ldcg(h_e + i) : __ldcg(cur + (uint64_t)i * nx + j + 4); };
        auto emit = [&](int i, const float4 &up, const float4 &mid, const float4 &dn, float lf, float rt) {
            float4 o;
            o.x = jac(up.x, dn.x, lf, mid.y);
            o.y = jac(up.y, dn.y, mid.x, mid.z);
            o.z = jac(up.z, dn.z, mid.y, mid.w);
            o.w = jac(up.w, dn.w, mid.z, rt);
            *reinterpret_cast<float4 *>(nxt + (uint64_t)i * nx + j) = o;
            if (send) {  // fused device-initiated puts of the new boundary
                if (i == 0) *reinterpret_cast<float4 *>(to_n + j) = o;
                if (i == ny - 1) *reinterpret_cast<float4 *>(to_s + j) = o;
                if (c4 == 0) to_w[i] = o.x;
                if (c4 == W4 - 1) to_e[i] = o.w;
            }
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

// The initial halos: tile[0]'s boundary into the neighbours' halo[0].
__device__ __forceinline__ void halo_prime(const HaloArgs &a, shmemg_group g, int me, const int nb[4]) {
    const shmemg_device_ctx_t &c = a.c;
    const int nx = a.nx, ny = a.ny;
    const float *t0 = (const float *)shmemg_d_addr(c, me, a.tiles);
    auto nb_halo = [&](int dir, int part) {
        return (float *)shmemg_d_addr(c, nb[dir], a.halos) +
               (part == H_N ? 0 : part == H_S ? nx : part == H_W ? 2 * nx : 2 * nx + ny);
    };
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

// Persistent form: the whole run in one cooperative launch, PEs synchronised pairwise by
// their signals only.
__global__ void __launch_bounds__(512) k_halo(HaloArgs a, int iters) {
    const shmemg_device_ctx_t &c = a.c;
    const int me = shmemg_d_my_pe(c);
    const shmemg_group g = shmemg_d_group_pe(c);
    const bool leader = shmemg_d_pe_leader(c);
    __shared__ int s_stop;
    int nb[4];
    halo_neighbours(a, me, nb);
    if (threadIdx.x == 0) s_stop = 0;
    halo_prime(a, g, me, nb);
    shmemg_d_pe_sync(c);
    if (leader) halo_signal(a, nb);
    uint64_t *my_sig = (uint64_t *)shmemg_d_addr(c, me, a.sigs);
    for (int t = 0; t < iters; t++) {
        if (threadIdx.x == 0) {
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
        const bool send = t + 1 < iters;
        halo_sweep(a, g, me, nb, t & 1, send);
        shmemg_d_pe_sync(c);
        if (send && leader) halo_signal(a, nb);
    }
    // every halo meant for this PE has arrived (or the run failed): reset the counters
    // for the next run
    shmemg_d_pe_sync(c);
    if (leader)
        for (int d = 0; d < 4; d++) my_sig[d] = 0;
}

// Launch-per-sweep form (the plain path): kernel boundaries order the sweeps, no signals.
__global__ void __launch_bounds__(512) k_halo_step(HaloArgs a, int t, int send, int prime) {
    const int me = shmemg_d_my_pe(a.c);
    const shmemg_group g = shmemg_d_group_pe(a.c);
    int nb[4];
    halo_neighbours(a, me, nb);
    if (prime) halo_prime(a, g, me, nb);
    else halo_sweep(a, g, me, nb, t & 1, send != 0);
}


// 512 threads per PE: one CTA of 512, or cluster_dim CTAs of 512 / cluster_dim (so a
// clustered PE spreads the same work over more SMs and every PE still fits at once)
static int halo_threads() {
    const State &S = st();
    return S.pe_mode == SHMEMG_PE_MODE_CLUSTER ? 512 / S.cluster_dim : 512;
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

extern "C" int shmemg_halo_jacobi(float *tiles, float *halos, uint64_t *sigs, int px, int py, int nx, int ny,
                                  int iters, void *stream) {
    HaloArgs a;
    if (int rc = halo_args(tiles, halos, sigs, px, py, nx, ny, iters, &a)) return rc;
    if (iters == 0) return SHMEMG_SUCCESS;
    void *args[] = {(void *)&a, (void *)&iters};
    return launch_pe_grid((const void *)k_halo, args, 0, to_stream(stream), halo_threads());
}

extern "C" int shmemg_halo_jacobi_plain(float *tiles, float *halos, uint64_t *sigs, int px, int py, int nx, int ny,
                                        int iters, void *stream) {
    HaloArgs a;
    if (int rc = halo_args(tiles, halos, sigs, px, py, nx, ny, iters, &a)) return rc;
    if (iters == 0) return SHMEMG_SUCCESS;
    int t = 0, send = 0, prime = 1;
    void *args[] = {(void *)&a, (void *)&t, (void *)&send, (void *)&prime};
    if (int rc = launch_pe_grid((const void *)k_halo_step, args, 0, to_stream(stream), halo_threads())) return rc;
    prime = 0;
    for (t = 0; t < iters; t++) {
        send = t + 1 < iters;
        if (int rc = launch_pe_grid((const void *)k_halo_step, args, 0, to_stream(stream), halo_threads())) return rc;
    }
    return SHMEMG_SUCCESS;
}
