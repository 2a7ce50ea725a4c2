// Parallel aggregation on the device: the coarsening step of Alg. 1
// ("construct P_i from A_i") with the point-wise aggregation of Sec. 4, its
// aggregates grown around a distance-2 maximal independent set (MIS-2) of
// the strong-connection graph instead of by the sequential greedy passes of
// the host aggregation.
//
// Graph: J != I is a neighbour of I when the strength flag of block (I, J)
// or of block (J, I) is set (the strong connections made undirected; the
// block pattern is symmetric, so (J, I) is found by a binary search in row J).
//
// Roots: each node carries a 64-bit key (state << 32 | priority), state 2 =
// root, 1 = undecided, 0 = excluded or without neighbours, priority =
// MurmurHash3's 32-bit finaliser of the node index (a bijection of 32-bit
// integers, so keys of equal state never tie).  One round:
//   max1[u] = the largest key over u and its neighbours,
//   max2[v] = the largest max1 over v and its neighbours
//           = the largest key within two edges of v;
// an undecided v whose own key equals max2[v] becomes a root, and one whose
// max2[v] is a root's key is excluded.  Rounds repeat until no node is
// undecided.  A node becomes a root exactly when, among the undecided nodes
// within two edges, it has the highest priority and no root lies within
// two edges, so the roots are those of the sequential visit of the nodes in
// descending priority (the greedy maximal independent set of the squared
// graph), whatever the round structure.
//
// Aggregates: a root and its neighbours, numbered in ascending root index
// (roots are at least three edges apart, so no node neighbours two roots);
// then every other node with a neighbour joins the aggregate of its
// lowest-index neighbour that has one (one exists because the root set is
// maximal).  Nodes without neighbours stay unaggregated (-1).
#include <algorithm>

#include "amg_internal.cuh"

namespace amg {

int exclusive_scan_i32(const int *in, int *out, int n, int *total_host, DevArena &tmp,
                       cudaStream_t s);

namespace {

constexpr int MT = 256;                       // threads per CTA: 8 warps, one node each
constexpr uint64_t KEY_ROOT = 2ull << 32;
constexpr uint64_t KEY_UNDECIDED = 1ull << 32;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t node_priority(uint32_t h)
{
    // MurmurHash3 fmix32 (Appleby): xor-shift / multiply avalanche rounds
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const uint64_t o = __shfl_xor_sync(FULL, v, m);
        v = o > v ? o : v;
    }
    return v;
}

__device__ __forceinline__ int warp_id_global() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int warps_in_grid() { return (gridDim.x * blockDim.x) >> 5; }

// link[p] = 1 when entry p = (I, J), J != I, is strong in either direction;
// key[I] = the initial key (undecided if I has a link, else excluded).
__global__ void __launch_bounds__(MT) mis2_links_kernel(const int *__restrict__ rp,
                                                        const int *__restrict__ col,
                                                        const uint8_t *__restrict__ strong,
                                                        int nn, uint8_t *__restrict__ link,
                                                        uint64_t *__restrict__ key)
{
    const int lane = threadIdx.x & 31;
    for (int I = warp_id_global(); I < nn; I += warps_in_grid()) {
        const int b = rp[I], e = rp[I + 1];
        unsigned any = 0;
        for (int base = b; base < e; base += 32) {
            const int p = base + lane;
            uint8_t l = 0;
            if (p < e) {
                const int J = col[p];
                if (J != I) {
                    l = strong[p];
                    if (!l) {
                        int lo = rp[J], hi = rp[J + 1];
                        const int end = hi;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (col[mid] < I) lo = mid + 1;
                            else hi = mid;
                        }
                        if (lo < end && col[lo] == I) l = strong[lo];
                    }
                }
                link[p] = l;
            }
            any |= __ballot_sync(FULL, l != 0);
        }
        if (lane == 0) key[I] = (any ? KEY_UNDECIDED : 0ull) | node_priority((uint32_t)I);
    }
}

// max1[u] = max(key[u], key[J] for linked J).
__global__ void __launch_bounds__(MT) mis2_max1_kernel(const int *__restrict__ rp,
                                                       const int *__restrict__ col,
                                                       const uint8_t *__restrict__ link,
                                                       const uint64_t *__restrict__ key, int nn,
                                                       uint64_t *__restrict__ max1)
{
    const int lane = threadIdx.x & 31;
    for (int u = warp_id_global(); u < nn; u += warps_in_grid()) {
        const int b = rp[u], e = rp[u + 1];
        uint64_t m = 0;
        for (int p = b + lane; p < e; p += 32)
            if (link[p]) {
                const uint64_t k = key[col[p]];
                m = k > m ? k : m;
            }
        m = warp_max_u64(m);
        if (lane == 0) {
            const uint64_t k = key[u];
            max1[u] = k > m ? k : m;
        }
    }
}

// For undecided v: max2 = max(max1[v], max1[J] for linked J); root when it
// is v's own key, excluded when it is a root's; otherwise v stays undecided
// and *undecided is set.
__global__ void __launch_bounds__(MT) mis2_max2_kernel(const int *__restrict__ rp,
                                                       const int *__restrict__ col,
                                                       const uint8_t *__restrict__ link,
                                                       const uint64_t *__restrict__ max1, int nn,
                                                       uint64_t *__restrict__ key,
                                                       int *__restrict__ undecided)
{
    const int lane = threadIdx.x & 31;
    for (int v = warp_id_global(); v < nn; v += warps_in_grid()) {
        const uint64_t k = key[v];
        if ((k >> 32) != 1) continue;  // warp-uniform
        const int b = rp[v], e = rp[v + 1];
        uint64_t m = 0;
        for (int p = b + lane; p < e; p += 32)
            if (link[p]) {
                const uint64_t t = max1[col[p]];
                m = t > m ? t : m;
            }
        m = warp_max_u64(m);
        if (lane == 0) {
            const uint64_t m1 = max1[v];
            m = m1 > m ? m1 : m;
            if (m == k) key[v] = KEY_ROOT | (k & 0xffffffffull);
            else if ((m >> 32) == 2) key[v] = k & 0xffffffffull;
            else *undecided = 1;
        }
    }
}

__global__ void mis2_root_flags_kernel(const uint64_t *__restrict__ key, int nn,
                                       int *__restrict__ is_root)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nn) is_root[v] = (key[v] >> 32) == 2 ? 1 : 0;
}

// step1[v] = id of v if v is a root, else the id of its root neighbour (-1
// if none); two root neighbours set bit 0 of *bad.
__global__ void __launch_bounds__(MT) mis2_step1_kernel(const int *__restrict__ rp,
                                                        const int *__restrict__ col,
                                                        const uint8_t *__restrict__ link,
                                                        const uint64_t *__restrict__ key,
                                                        const int *__restrict__ id, int nn,
                                                        int *__restrict__ step1,
                                                        int *__restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    for (int v = warp_id_global(); v < nn; v += warps_in_grid()) {
        if ((key[v] >> 32) == 2) {
            if (lane == 0) step1[v] = id[v];
            continue;
        }
        const int b = rp[v], e = rp[v + 1];
        int found = -1, count = 0;
        for (int base = b; base < e; base += 32) {
            const int p = base + lane;
            const bool r = p < e && link[p] && (key[col[p]] >> 32) == 2;
            const unsigned bal = __ballot_sync(FULL, r);
            count += __popc(bal);
            if (bal && found < 0) found = id[col[base + __ffs(bal) - 1]];
        }
        if (lane == 0) {
            step1[v] = count ? found : -1;
            if (count > 1) atomicOr(bad, 1);
        }
    }
}

// agg[v] = step1[v] if set; else the step1 of the lowest-index linked
// neighbour that has one; -1 for nodes without links.  A linked node left
// without an aggregate sets bit 1 of *bad.
__global__ void __launch_bounds__(MT) mis2_step2_kernel(const int *__restrict__ rp,
                                                        const int *__restrict__ col,
                                                        const uint8_t *__restrict__ link,
                                                        const int *__restrict__ step1, int nn,
                                                        int *__restrict__ agg,
                                                        int *__restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    for (int v = warp_id_global(); v < nn; v += warps_in_grid()) {
        const int s1 = step1[v];
        if (s1 >= 0) {
            if (lane == 0) agg[v] = s1;
            continue;
        }
        const int b = rp[v], e = rp[v + 1];
        int found = -1;
        unsigned any = 0;
        for (int base = b; base < e && found < 0; base += 32) {
            const int p = base + lane;
            const bool l = p < e && link[p];
            any |= __ballot_sync(FULL, l);
            const unsigned bal = __ballot_sync(FULL, l && step1[col[p]] >= 0);
            if (bal) found = step1[col[base + __ffs(bal) - 1]];
        }
        if (lane == 0) {
            agg[v] = found;
            if (found < 0 && any) atomicOr(bad, 2);
        }
    }
}

}  // namespace

int aggregate_mis2(const BsrD &A, const uint8_t *strong, int *agg, int *nagg_host, int *rounds_host,
                   DevArena &tmp, cudaStream_t s)
{
    const int nn = A.nbr;
    *nagg_host = 0;
    if (rounds_host) *rounds_host = 0;
    if (nn == 0) return AMG_OK;
    if (A.nbc != nn) {
        set_error("MIS-2 aggregation needs a square block pattern");
        return AMG_ERR_ARG;
    }
    uint8_t *link = nullptr;
    uint64_t *key = nullptr, *max1 = nullptr;
    int *flags = nullptr, *is_root = nullptr, *id = nullptr, *step1 = nullptr;
    AMG_TRY(tmp.alloc_n(&link, (size_t)std::max<int64_t>(A.nnzb, 1)));
    AMG_TRY(tmp.alloc_n(&key, (size_t)nn));
    AMG_TRY(tmp.alloc_n(&max1, (size_t)nn));
    AMG_TRY(tmp.alloc_n(&flags, 2));  // [0] undecided, [1] bad
    AMG_TRY(tmp.alloc_n(&is_root, (size_t)nn));
    AMG_TRY(tmp.alloc_n(&id, (size_t)nn + 1));
    AMG_TRY(tmp.alloc_n(&step1, (size_t)nn));
    Geom g;
    AMG_TRY(query_geom(&g));
    const int grid = (int)std::min<int64_t>(((int64_t)nn + 7) / 8, (int64_t)g.num_sms * 16);
    mis2_links_kernel<<<grid, MT, 0, s>>>(A.row_ptr, A.col, strong, nn, link, key);
    ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    // every round decides at least the undecided node of highest priority
    int rounds = 0;
    for (;;) {
        AMG_TRY_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), s));
        mis2_max1_kernel<<<grid, MT, 0, s>>>(A.row_ptr, A.col, link, key, nn, max1);
        mis2_max2_kernel<<<grid, MT, 0, s>>>(A.row_ptr, A.col, link, max1, nn, key, flags);
        ::amg::count_launch(2);
        AMG_TRY_CUDA(cudaGetLastError());
        ++rounds;
        int und = 0;
        AMG_TRY_CUDA(cudaMemcpyAsync(&und, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        if (!und) break;
        if (rounds > nn) {
            set_error("MIS-2 aggregation did not settle in %d rounds", rounds);
            return AMG_ERR_STATE;
        }
    }
    mis2_root_flags_kernel<<<(nn + 255) / 256, 256, 0, s>>>(key, nn, is_root);
    ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    int nagg = 0;
    AMG_TRY(exclusive_scan_i32(is_root, id, nn, &nagg, tmp, s));
    AMG_TRY_CUDA(cudaMemsetAsync(flags + 1, 0, sizeof(int), s));
    mis2_step1_kernel<<<grid, MT, 0, s>>>(A.row_ptr, A.col, link, key, id, nn, step1, flags + 1);
    mis2_step2_kernel<<<grid, MT, 0, s>>>(A.row_ptr, A.col, link, step1, nn, agg, flags + 1);
    ::amg::count_launch(2);
    AMG_TRY_CUDA(cudaGetLastError());
    int bad = 0;
    AMG_TRY_CUDA(cudaMemcpyAsync(&bad, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    tmp.release(step1);
    tmp.release(id);
    tmp.release(is_root);
    tmp.release(flags);
    tmp.release(max1);
    tmp.release(key);
    tmp.release(link);
    if (bad) {
        set_error("MIS-2 aggregation: %s", (bad & 1) ? "a node neighbours two roots"
                                                     : "a linked node was left unaggregated");
        return AMG_ERR_STATE;
    }
    *nagg_host = nagg;
    if (rounds_host) *rounds_host = rounds;
    return AMG_OK;
}

}  // namespace amg
