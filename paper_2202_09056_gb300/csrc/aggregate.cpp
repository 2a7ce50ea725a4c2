// Host-side greedy aggregation on the strong-connection graph of a block
// matrix: the coarsening step of Alg. 1 ("construct P_i from A_i"), with the
// point-wise (node = block row) aggregation of Sec. 4.  The graph is tiny
// next to the matrix values and the passes are inherently sequential, so
// this one step of the setup runs on the host; the strength flags come from
// the device and the aggregate map goes back to it.
//
// Three passes over the nodes in ascending order:
//   1. a free node all of whose strong neighbours are free becomes the root
//      of a new aggregate holding itself and those neighbours;
//   2. a node still free joins the aggregate of its lowest-numbered strong
//      neighbour that was placed in pass 1;
//   3. a node still free starts a new aggregate with its free strong
//      neighbours.
// Nodes with no strong neighbour are isolated (-1): no aggregate, zero row
// in the prolongation.  Aggregates are numbered in creation order.
#include <cstdint>
#include <vector>

#include "../../include/amg_gb300.h"

namespace amg {

int aggregate_host(int nn, const int *row_ptr, const int *col, const uint8_t *strong, int *agg,
                   int *nagg)
{
    constexpr int kUnassigned = -1;
    constexpr int kLonely = -2;
    std::vector<char> root_pass(nn, 0);  // placed during pass 1
    for (int node = 0; node < nn; ++node) {
        int links = 0;
        for (int e = row_ptr[node]; e < row_ptr[node + 1]; ++e) links += strong[e] ? 1 : 0;
        agg[node] = links ? kUnassigned : kLonely;
    }
    int count = 0;
    for (int node = 0; node < nn; ++node) {  // pass 1
        if (agg[node] != kUnassigned) continue;
        bool neighbourhood_free = true;
        for (int e = row_ptr[node]; e < row_ptr[node + 1] && neighbourhood_free; ++e)
            if (strong[e] && agg[col[e]] != kUnassigned) neighbourhood_free = false;
        if (!neighbourhood_free) continue;
        agg[node] = count;
        root_pass[node] = 1;
        for (int e = row_ptr[node]; e < row_ptr[node + 1]; ++e)
            if (strong[e]) {
                agg[col[e]] = count;
                root_pass[col[e]] = 1;
            }
        ++count;
    }
    for (int node = 0; node < nn; ++node) {  // pass 2
        if (agg[node] != kUnassigned) continue;
        for (int e = row_ptr[node]; e < row_ptr[node + 1]; ++e)
            if (strong[e] && root_pass[col[e]]) {
                agg[node] = agg[col[e]];
                break;
            }
    }
    for (int node = 0; node < nn; ++node) {  // pass 3
        if (agg[node] != kUnassigned) continue;
        agg[node] = count;
        for (int e = row_ptr[node]; e < row_ptr[node + 1]; ++e)
            if (strong[e] && agg[col[e]] == kUnassigned) agg[col[e]] = count;
        ++count;
    }
    for (int node = 0; node < nn; ++node)
        if (agg[node] == kLonely) agg[node] = -1;
    *nagg = count;
    return AMG_OK;
}

}  // namespace amg
