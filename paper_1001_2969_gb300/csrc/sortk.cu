// sortk.cu -- the per-step cell sort of the particle store and the canonical
// numbering of newborn particles.
//
// Cell sort: counts per cell (made by the particle pass), an exclusive scan
// into per-cell cursors, then a rank pass that writes the permutation the
// next pass reads through.  Dead particles (cell -1) are left out, so the
// sort also compacts.  Order inside a cell is not fixed (shared and global
// atomics hand out the places).
//
// Newborns are numbered next_id + stride x rank of their key (parent
// species, parent id, birth slot; the stride is 1 unless the reactor's
// particles are shared among processes): one block ranks small batches directly, larger batches
// go through an LSD radix sort of (key, index) pairs, both in one
// cooperative launch that reads the count on the device.
#include <limits.h>

#include <algorithm>

#include "pic_internal.cuh"

namespace pic {

template <typename T>
__global__ void k_hist(PBuf<T> buf, const int32_t *n_dev, int32_t *counts) {
    const int n = *n_dev;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int k = base + threadIdx.x;
        const int c = k < n ? buf.cell[k] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && lane == __ffs(peers) - 1) atomicAdd(counts + c, __popc(peers));
    }
}

template <typename T>
void launch_hist(PBuf<T> buf, const int32_t *n_dev, int32_t *counts, cudaStream_t st) {
    k_hist<T><<<152 * 8, 256, 0, st>>>(buf, n_dev, counts);
}

// ---- exclusive scan over cells: tiles of 4096 (1024 threads x 4) ----
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 4096;

__device__ __forceinline__ int block_exclusive_scan(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int warp_excl = warp > 0 ? s_warp[warp - 1] : 0;
    if (total) *total = s_warp[(blockDim.x >> 5) - 1];
    return warp_excl + x - v;
}

__global__ void k_scan_tiles(const int32_t *counts, int ncell, int32_t *block_sums, const StepCtl *ctl) {
    __shared__ int s_warp[32];
    if (sort_skip(ctl)) return;
    const int base = blockIdx.x * kScanTile + threadIdx.x * 4;
    int v = 0;
    for (int q = 0; q < 4; ++q) v += (base + q < ncell) ? counts[base + q] : 0;
    int tot;
    block_exclusive_scan(v, s_warp, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(int32_t *block_sums, int nblocks, int32_t *n_alive, int64_t capacity,
                           DevScalars *ds, const StepCtl *ctl) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (sort_skip(ctl)) return;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += blockDim.x) {
        const int k = b0 + threadIdx.x;
        const int v = k < nblocks ? block_sums[k] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, s_warp, &tot);
        const int carry = s_carry;
        if (k < nblocks) block_sums[k] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *n_alive = s_carry;
        if ((int64_t)s_carry > capacity) atomicOr(&ds->status, ST_CAPACITY);
    }
}

__global__ void k_scan_apply(const int32_t *counts, int ncell, const int32_t *block_sums,
                             int32_t *cursor, const StepCtl *ctl) {
    __shared__ int s_warp[32];
    if (sort_skip(ctl)) return;
    const int base = blockIdx.x * kScanTile + threadIdx.x * 4;
    int c[4];
    int v = 0;
    for (int q = 0; q < 4; ++q) {
        c[q] = (base + q < ncell) ? counts[base + q] : 0;
        v += c[q];
    }
    int ex = block_exclusive_scan(v, s_warp, nullptr) + block_sums[blockIdx.x];
    for (int q = 0; q < 4; ++q) {
        if (base + q < ncell) cursor[base + q] = ex;
        ex += c[q];
    }
}

// the whole scan in one block (meshes of at most kScanOne cells, a batch's
// small reactors): each thread sums a run of consecutive cells, one block
// scan, then each thread writes its run's cursors.  Larger meshes take the
// three tile kernels, whose loads coalesce.
constexpr int kScanOne = 16384;
__global__ void __launch_bounds__(kScanThreads)
    k_scan_one(const int32_t *counts, int ncell, int32_t *cursor, int32_t *n_alive, int64_t capacity,
               DevScalars *ds, const StepCtl *ctl) {
    __shared__ int s_warp[32];
    if (sort_skip(ctl)) return;
    const int per = (ncell + kScanThreads - 1) / kScanThreads;
    const int c0 = min(ncell, threadIdx.x * per), c1 = min(ncell, c0 + per);
    int v = 0;
    for (int c = c0; c < c1; ++c) v += counts[c];
    int tot;
    int ex = block_exclusive_scan(v, s_warp, &tot);
    for (int c = c0; c < c1; ++c) {
        const int x = counts[c];
        cursor[c] = ex;
        ex += x;
    }
    if (threadIdx.x == 0) {
        *n_alive = tot;
        if ((int64_t)tot > capacity) atomicOr(&ds->status, ST_CAPACITY);
    }
}

void launch_scan(const int32_t *counts, int32_t *cursor, int ncell, int32_t *block_sums,
                 int32_t *n_alive, int64_t capacity, DevScalars *ds, const StepCtl *ctl,
                 cudaStream_t st) {
    if (ncell <= kScanOne) {
        k_scan_one<<<1, kScanThreads, 0, st>>>(counts, ncell, cursor, n_alive, capacity, ds, ctl);
        return;
    }
    const int nb = (ncell + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<nb, kScanThreads, 0, st>>>(counts, ncell, block_sums, ctl);
    k_scan_top<<<1, kScanThreads, 0, st>>>(block_sums, nb, n_alive, capacity, ds, ctl);
    k_scan_apply<<<nb, kScanThreads, 0, st>>>(counts, ncell, block_sums, cursor, ctl);
}

__global__ void k_step_check(const DevScalars *ds, StepCtl *ctl) {
    if (sort_skip(ctl)) return;
    const int st = ds->status & (ST_CAPACITY | ST_BIRTH_OVERFLOW);
    if (st) sort_failed(ctl, st);
}

void launch_step_check(const DevScalars *ds, StepCtl *ctl, cudaStream_t st) {
    k_step_check<<<1, 1, 0, st>>>(ds, ctl);
}

// ---- rank: perm[cursor[cell]++] = element (main first, then births) ----
//
// A block takes segments of kRankSeg consecutive elements.  The main set is
// in (old) cell order and a particle moves at most a few cells per step, so
// the new cells of a segment fall in a window of at most kRankWin cells above
// the segment's smallest: the block counts its elements per window cell in
// shared memory (the count a shared atomic returns is the element's rank in
// the block), reserves each cell's places with one global atomic per
// distinct cell, and writes the permutation.  A segment whose cells spread
// wider (the births, which come in any order) ranks warp by warp: one
// global atomic per distinct cell of a warp (__match_any_sync).
constexpr int kRankThreads = 256;
constexpr int kRankPer = 8;
constexpr int kRankSeg = kRankThreads * kRankPer;
constexpr int kRankWin = 2048;

template <typename T>
__global__ void __launch_bounds__(kRankThreads)
    k_rank(PBuf<T> mainb, const int32_t *n_main_dev, PBuf<T> births, const int32_t *n_births_dev,
           int32_t *cursor, int32_t *perm, const int32_t *n_alive, int64_t cap, const int32_t *status,
           const StepCtl *ctl, int ncell) {
    __shared__ int s_hist[kRankWin];
    __shared__ int s_lo, s_hi;
    // a failed step keeps the previous permutation
    if (sort_skip(ctl) || (int64_t)*n_alive > cap || (*status & (ST_CAPACITY | ST_BIRTH_OVERFLOW))) return;
    const int nm = *n_main_dev, nb = *n_births_dev;
    const int total = nm + nb;
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    // the cells of a segment; the next segment's are requested before the
    // current one is ranked
    auto load = [&](int base, int *c) {
#pragma unroll
        for (int u = 0; u < kRankPer; ++u) {
            const int e = base + u * kRankThreads + tid;
            int v = -1;
            if (e < nm)
                v = mainb.cell[e];
            else if (e < total)
                v = births.cell[e - nm];
            c[u] = v < ncell ? v : -1;  // never a cell of the mesh: no place is taken for it
        }
    };
    int c[kRankPer];
    load(blockIdx.x * kRankSeg, c);
    for (int seg = blockIdx.x; seg * kRankSeg < total; seg += gridDim.x) {
        const int base = seg * kRankSeg;
        int lo = INT_MAX, hi = -1;
#pragma unroll
        for (int u = 0; u < kRankPer; ++u)
            if (c[u] >= 0) {
                lo = min(lo, c[u]);
                hi = max(hi, c[u]);
            }
        if (tid == 0) {
            s_lo = INT_MAX;
            s_hi = -1;
        }
        __syncthreads();
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0) {
            atomicMin(&s_lo, lo);
            atomicMax(&s_hi, hi);
        }
        __syncthreads();
        const int wlo = s_lo, whi = s_hi;
        int cn[kRankPer];
        load(base + gridDim.x * kRankSeg, cn);
        if (whi >= 0 && whi - wlo < kRankWin) {
            for (int w = tid; w <= whi - wlo; w += kRankThreads) s_hist[w] = 0;
            __syncthreads();
            // rank inside the block: lanes of a warp with one cell share one
            // shared atomic (an ion warp is mostly a single cell)
            int r[kRankPer];
#pragma unroll
            for (int u = 0; u < kRankPer; ++u) {
                const unsigned peers = __match_any_sync(0xffffffffu, c[u]);
                const int first = __ffs(peers) - 1;
                int b = 0;
                if (c[u] >= 0 && lane == first) b = atomicAdd(&s_hist[c[u] - wlo], __popc(peers));
                r[u] = __shfl_sync(0xffffffffu, b, first) + __popc(peers & lt);
            }
            __syncthreads();
            // each cell's places: one global atomic per distinct cell
            for (int w = tid; w <= whi - wlo; w += kRankThreads) {
                const int k = s_hist[w];
                if (k > 0) s_hist[w] = atomicAdd(cursor + wlo + w, k);
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kRankPer; ++u) {
                if (c[u] < 0) continue;
                const int pos = s_hist[c[u] - wlo] + r[u];
                // (cells and counts agree, so pos < *n_alive <= cap; the bound
                // keeps an inconsistent pass from writing past the permutation)
                if ((int64_t)pos < cap) perm[pos] = base + u * kRankThreads + tid;
            }
        } else if (whi >= 0) {
#pragma unroll
            for (int u = 0; u < kRankPer; ++u) {
                const unsigned peers = __match_any_sync(0xffffffffu, c[u]);
                const int first = __ffs(peers) - 1;
                int pos = 0;
                if (c[u] >= 0 && lane == first) pos = atomicAdd(cursor + c[u], __popc(peers));
                pos = __shfl_sync(0xffffffffu, pos, first) + __popc(peers & lt);
                if (c[u] >= 0 && (int64_t)pos < cap) perm[pos] = base + u * kRankThreads + tid;
            }
        }
        __syncthreads();  // s_lo, s_hi and s_hist are reused by the next segment
#pragma unroll
        for (int u = 0; u < kRankPer; ++u) c[u] = cn[u];
    }
}

template <typename T>
void launch_rank(PBuf<T> mainb, const int32_t *n_main, PBuf<T> births, const int32_t *n_births,
                 int32_t *cursor, int32_t *perm, const int32_t *n_alive, int64_t cap,
                 const int32_t *status, const StepCtl *ctl, int ncell, cudaStream_t st) {
    // a few segments per block: beside the field solve the blocks retire
    // often, so the solve's blocks find SMs early; a small store takes no
    // more blocks than its capacity fills (blocks stride on)
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(152 * 8, (cap + kRankSeg - 1) / kRankSeg));
    k_rank<T><<<grid, kRankThreads, 0, st>>>(mainb, n_main, births, n_births, cursor, perm, n_alive, cap, status,
                                             ctl, ncell);
}

// ---- newborn numbering ----
// Births get ids next_id + rank of their key (parent species, parent id,
// birth index), as in the oracle.  One cooperative launch: up to
// kSmallBirths keys block 0 ranks each key by counting smaller ones; above
// that the grid runs an LSD radix sort over 8-bit digits (a digit shared by
// every key is skipped), tiles of kRadixTile keys, grid barriers between the
// histogram, scan and scatter phases.
constexpr int kSmallBirths = 2048;
constexpr int kRadixThreads = 1024;
constexpr int kRadixPer = 2;
constexpr int kRadixTile = kRadixThreads * kRadixPer;

__global__ void __launch_bounds__(kRadixThreads)
    k_birth_ids(const uint64_t *key, uint64_t *id, const int32_t *nb_dev, const int32_t *nb0_dev, StepCtl *ctl, int s,
                RadixTmp t) {
    // the small path's keys and the scatter's per-warp digit counts share space
    constexpr int kBuf = kSmallBirths * 8 > (kRadixThreads / 32) * 256 * 4 ? kSmallBirths * 8
                                                                            : (kRadixThreads / 32) * 256 * 4;
    __shared__ __align__(16) unsigned char s_buf[kBuf];
    uint64_t *s_key = reinterpret_cast<uint64_t *>(s_buf);
    uint32_t (*s_wc)[256] = reinterpret_cast<uint32_t (*)[256]>(s_buf);
    __shared__ uint32_t s_run[256];
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (sort_skip(ctl)) return;
    // the births of the last pass: the buffer's entries from *nb0_dev on
    const int first = nb0_dev ? *nb0_dev : 0;
    const int nb = *nb_dev - first;
    if (nb <= 0 || first < 0) return;
    key += first;
    id += first;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (nb <= kSmallBirths) {
        if (blockIdx.x != 0) return;
        const uint64_t base = ctl->next_id[s];
        const uint64_t stride = ctl->id_stride ? ctl->id_stride : 1ull;
        for (int k = tid; k < nb; k += blockDim.x) s_key[k] = key[k];
        __syncthreads();
        for (int k = tid; k < nb; k += blockDim.x) {
            const uint64_t mine = s_key[k];
            int rank = 0;
            for (int q = 0; q < nb; ++q) rank += s_key[q] < mine;
            id[k] = base + stride * (uint64_t)rank;
        }
        __syncthreads();
        if (tid == 0) ctl->next_id[s] = base + stride * (uint64_t)nb;
        return;
    }
    // every block reads the base before the first barrier; block 0 moves it on at the end
    const uint64_t base = ctl->next_id[s];
    const uint64_t stride = ctl->id_stride ? ctl->id_stride : 1ull;
    const int ntiles = (nb + kRadixTile - 1) / kRadixTile;
    unsigned nbar = 0;
    // a wait that gives up fails the sort (its ids would be wrong)
    auto bar = [&]() {
        if (count_barrier(&ctl->bar, (++nbar) * gridDim.x, &ctl->bar_timeout)) return true;
        if (tid == 0) sort_failed(ctl, ST_TIMEOUT);
        return false;
    };
    for (int e = blockIdx.x * blockDim.x + tid; e < nb; e += gridDim.x * blockDim.x) {
        t.k0[e] = key[e];
        t.v0[e] = (uint32_t)e;
    }
    if (!bar()) return;
    uint64_t *ka = t.k0, *kb = t.k1;
    uint32_t *va = t.v0, *vb = t.v1;
    for (int shift = 0; shift < 64; shift += 8) {
        // digit histogram per tile: hist[d * ntiles + tile]
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if (tid < 256) s_run[tid] = 0;
            __syncthreads();
            for (int q = 0; q < kRadixPer; ++q) {
                const int e = tile * kRadixTile + q * kRadixThreads + tid;
                if (e < nb) atomicAdd(&s_run[(ka[e] >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (tid < 256) t.hist[tid * ntiles + tile] = s_run[tid];
            __syncthreads();
        }
        if (!bar()) return;
        // block 0: exclusive scan in digit-major order; a digit held by all
        // keys leaves the order as it is
        if (blockIdx.x == 0) {
            if (tid < 256) {
                uint32_t c = 0;
                for (int tl = 0; tl < ntiles; ++tl) c += t.hist[tid * ntiles + tl];
                s_run[tid] = c;
            }
            __syncthreads();
            int all = 0;
            for (int d = 0; d < 256; ++d) all |= s_run[d] == (uint32_t)nb;
            if (tid == 0) *t.flag = all;
            if (!all) {
                if (tid == 0) s_carry = 0;
                __syncthreads();
                const int total = 256 * ntiles;
                for (int b0 = 0; b0 < total; b0 += blockDim.x) {
                    const int k = b0 + tid;
                    const int v = k < total ? (int)t.hist[k] : 0;
                    int tot;
                    const int ex = block_exclusive_scan(v, s_warp, &tot);
                    const int carry = s_carry;
                    if (k < total) t.hist[k] = (uint32_t)(carry + ex);
                    __syncthreads();
                    if (tid == 0) s_carry = carry + tot;
                    __syncthreads();
                }
            }
        }
        if (!bar()) return;
        if (*(volatile int *)t.flag) continue;
        // stable scatter of each tile: rounds of kRadixThreads keys in order;
        // inside a round a key's place is (keys of its digit in earlier
        // warps) + (earlier lanes of its warp with the same digit)
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if (tid < 256) s_run[tid] = t.hist[tid * ntiles + tile];
            for (int k = tid; k < (kRadixThreads / 32) * 256; k += blockDim.x) (&s_wc[0][0])[k] = 0;
            __syncthreads();
            for (int q = 0; q < kRadixPer; ++q) {
                const int e = tile * kRadixTile + q * kRadixThreads + tid;
                const bool valid = e < nb;
                const uint64_t kv = valid ? ka[e] : 0;
                const int d = valid ? (int)((kv >> shift) & 255u) : 256 + lane;  // unique dummies
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                const int rank_w = __popc(peers & ((1u << lane) - 1u));
                if (valid && lane == __ffs(peers) - 1) s_wc[warp][d] = __popc(peers);
                __syncthreads();
                if (valid) {
                    uint32_t off = s_run[d];
                    for (int w = 0; w < warp; ++w) off += s_wc[w][d];
                    const uint32_t pos = off + (uint32_t)rank_w;
                    kb[pos] = kv;
                    vb[pos] = va[e];
                }
                __syncthreads();
                if (tid < 256) {
                    uint32_t add = 0;
                    for (int w = 0; w < kRadixThreads / 32; ++w) {
                        add += s_wc[w][tid];
                        s_wc[w][tid] = 0;
                    }
                    s_run[tid] += add;
                }
                __syncthreads();
            }
        }
        if (!bar()) return;
        uint64_t *tk = ka;
        ka = kb;
        kb = tk;
        uint32_t *tv = va;
        va = vb;
        vb = tv;
    }
    for (int r = blockIdx.x * blockDim.x + tid; r < nb; r += gridDim.x * blockDim.x) id[va[r]] = base + stride * (uint64_t)r;
    if (blockIdx.x == 0 && tid == 0) ctl->next_id[s] = base + stride * (uint64_t)nb;
}

// failure-detection self-test: one block waits at the bounded grid barrier
// for a second participant that is never launched; the wait must give up
__global__ void k_wait_selftest(unsigned *count, int *timeout, long long limit, int *gave_up) {
    const bool ok = count_barrier(count, 2u, timeout, limit);
    if (threadIdx.x == 0) *gave_up = ok ? 0 : 1;
}

int wait_selftest(long long limit, int *gave_up) {
    int *buf = nullptr;  // count, timeout, result
    if (cudaMalloc(&buf, 3 * sizeof(int)) != cudaSuccess) return -1;
    cudaMemset(buf, 0, 3 * sizeof(int));
    k_wait_selftest<<<1, 32>>>(reinterpret_cast<unsigned *>(buf), buf + 1, limit, buf + 2);
    int out[3] = {0, 0, 0};
    const cudaError_t e = cudaMemcpy(out, buf, sizeof(out), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return -1;
    *gave_up = out[2] && out[1];
    return 0;
}

void launch_birth_ids(const uint64_t *key, uint64_t *id, const int32_t *nb, const int32_t *nb0, StepCtl *ctl,
                      int s, RadixTmp tmp, cudaStream_t st, int max_grid) {
    // one block per SM (the launch needs them co-resident), per device
    static int grids[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int &grid = grids[dev & 63];
    if (grid == 0) {
        int nsm = 0, per = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_birth_ids, kRadixThreads, 0);
        grid = std::max(1, std::min(nsm, nsm * per));
    }
    cudaMemsetAsync(&ctl->bar, 0, sizeof(unsigned) + sizeof(int32_t), st);  // counter and timeout flag
    void *args[] = {(void *)&key, (void *)&id, (void *)&nb, (void *)&nb0, (void *)&ctl, (void *)&s, (void *)&tmp};
    // no more blocks than tiles of the largest batch of births (a small
    // reactor's numbering does not hold the whole GPU)
    // (max_grid: a reactor of a batch, whose numbering must not wait for
    // many co-resident blocks while the other reactors' kernels hold SMs)
    const int g = std::max(1, std::min(std::min(grid, max_grid), (tmp.max_n + kRadixTile - 1) / kRadixTile));
    if (g == 1)  // one block: its barriers wait for itself alone, no co-residency to ask for
        k_birth_ids<<<1, kRadixThreads, 0, st>>>(key, id, nb, nb0, ctl, s, tmp);
    else
        cudaLaunchCooperativeKernel((void *)k_birth_ids, g, kRadixThreads, args, 0, st);
}

template void launch_hist<float>(PBuf<float>, const int32_t *, int32_t *, cudaStream_t);
template void launch_hist<double>(PBuf<double>, const int32_t *, int32_t *, cudaStream_t);
template void launch_rank<float>(PBuf<float>, const int32_t *, PBuf<float>, const int32_t *,
                                 int32_t *, int32_t *, const int32_t *, int64_t, const int32_t *,
                                 const StepCtl *, int, cudaStream_t);
template void launch_rank<double>(PBuf<double>, const int32_t *, PBuf<double>, const int32_t *,
                                  int32_t *, int32_t *, const int32_t *, int64_t, const int32_t *,
                                  const StepCtl *, int, cudaStream_t);

}  // namespace pic
