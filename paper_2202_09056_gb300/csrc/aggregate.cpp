// Host-side greedy aggregation on the strong-connection graph of a block
// matrix: the coarsening step of Alg. 1 ("construct P_i from A_i"), with the
// point-wise (node = block row) aggregation of Sec. 4.  The passes are
// inherently sequential, so this one step of the setup runs on the host; the
// device sends each node's strong neighbours (column order) and the
// aggregate map goes back to it.
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

// srp[nn + 1], scol: node i's strong neighbours are scol[srp[i] .. srp[i+1])
int aggregate_host(int nn, const int *srp, const int *scol, int *agg, int *nagg)
{
    constexpr int kUnassigned = -1;
    constexpr int kLonely = -2;
    std::vector<char> root_pass(nn, 0);  // placed during pass 1
    for (int node = 0; node < nn; ++node) agg[node] = srp[node + 1] > srp[node] ? kUnassigned : kLonely;
    int count = 0;
    for (int node = 0; node < nn; ++node) {  // pass 1
        if (agg[node] != kUnassigned) continue;
        bool neighbourhood_free = true;
        for (int e = srp[node]; e < srp[node + 1] && neighbourhood_free; ++e)
            if (agg[scol[e]] != kUnassigned) neighbourhood_free = false;
        if (!neighbourhood_free) continue;
        agg[node] = count;
        root_pass[node] = 1;
        for (int e = srp[node]; e < srp[node + 1]; ++e) {
            agg[scol[e]] = count;
            root_pass[scol[e]] = 1;
        }
        ++count;
    }
    for (int node = 0; node < nn; ++node) {  // pass 2
        if (agg[node] != kUnassigned) continue;
        for (int e = srp[node]; e < srp[node + 1]; ++e)
            if (root_pass[scol[e]]) {
                agg[node] = agg[scol[e]];
                break;
            }
    }
    for (int node = 0; node < nn; ++node) {  // pass 3
        if (agg[node] != kUnassigned) continue;
        agg[node] = count;
        for (int e = srp[node]; e < srp[node + 1]; ++e)
            if (agg[scol[e]] == kUnassigned) agg[scol[e]] = count;
        ++count;
    }
    for (int node = 0; node < nn; ++node)
        if (agg[node] == kLonely) agg[node] = -1;
    *nagg = count;
    return AMG_OK;
}

}  // namespace amg
