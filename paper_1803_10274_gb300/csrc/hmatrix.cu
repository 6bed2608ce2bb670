// Block partition of an H matrix over the cluster tree (paper Section 3.2,
// the H matrix representation: only well-separated sub-blocks are compressed,
// strong admissibility).  Host code: it needs no context and no GPU.
//
// A pair of nodes (t, s) is admissible when their bounding boxes are apart
// and min(diam t, diam s) <= eta dist(t, s) (diam: the box's diagonal;
// dist: Euclidean distance between the boxes; both summed coordinate by
// coordinate in order, then one correctly rounded square root).  From
// (root, root) an admissible pair is a far block, two leaves a near block,
// and any other pair is split into its children's pairs (both nodes when
// both have children, else the inner one), depth first, left child first.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace krr {
namespace {

double box_diam(const double *lo, const double *hi, int d, int v) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        const double g = hi[int64_t(v) * d + k] - lo[int64_t(v) * d + k];
        acc += g * g;
    }
    return std::sqrt(acc);
}

double box_dist(const double *lo, const double *hi, int d, int t, int s) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        const double a = lo[int64_t(s) * d + k] - hi[int64_t(t) * d + k];
        const double b = lo[int64_t(t) * d + k] - hi[int64_t(s) * d + k];
        const double g = std::fmax(0.0, std::fmax(a, b));
        acc += g * g;
    }
    return std::sqrt(acc);
}

}  // namespace
}  // namespace krr

extern "C" int krr_h_partition(int32_t n_nodes, const int32_t *left, const int32_t *right, int32_t d,
                               const double *lo, const double *hi, double eta, int32_t *near, int64_t cap_near,
                               int64_t *n_near, int32_t *far, int64_t cap_far, int64_t *n_far) {
    using namespace krr;
    if (n_nodes < 1 || d < 1 || !left || !right || !lo || !hi || !n_near || !n_far || !(eta >= 0.0) ||
        cap_near < 0 || cap_far < 0 || (cap_near > 0 && !near) || (cap_far > 0 && !far))
        return fail(KRR_ERR_INVALID_ARG, "krr_h_partition: bad arguments");
    // the tree: every inner node has two children of lower postorder id
    for (int32_t v = 0; v < n_nodes; ++v) {
        const int32_t l = left[v], r = right[v];
        if ((l < 0) != (r < 0) || (l >= 0 && (l >= v || r >= v)))
            return fail(KRR_ERR_INVALID_ARG, "krr_h_partition: not a binary tree in postorder");
    }
    std::vector<double> diam(n_nodes);
    for (int32_t v = 0; v < n_nodes; ++v) diam[v] = box_diam(lo, hi, d, v);
    int64_t nn = 0, nf = 0;
    // explicit stack of pairs, popped in the recursion's order
    std::vector<std::pair<int32_t, int32_t>> stack;
    stack.emplace_back(n_nodes - 1, n_nodes - 1);
    while (!stack.empty()) {
        const auto [t, s] = stack.back();
        stack.pop_back();
        const double dd = box_dist(lo, hi, d, t, s);
        if (dd > 0.0 && std::fmin(diam[t], diam[s]) <= eta * dd) {
            if (nf < cap_far) {
                far[2 * nf] = t;
                far[2 * nf + 1] = s;
            }
            ++nf;
            continue;
        }
        const bool tl = left[t] < 0, sl = left[s] < 0;
        if (tl && sl) {
            if (nn < cap_near) {
                near[2 * nn] = t;
                near[2 * nn + 1] = s;
            }
            ++nn;
        } else if (tl) {
            stack.emplace_back(t, right[s]);
            stack.emplace_back(t, left[s]);
        } else if (sl) {
            stack.emplace_back(right[t], s);
            stack.emplace_back(left[t], s);
        } else {  // visited (lt, ls), (lt, rs), (rt, ls), (rt, rs)
            stack.emplace_back(right[t], right[s]);
            stack.emplace_back(right[t], left[s]);
            stack.emplace_back(left[t], right[s]);
            stack.emplace_back(left[t], left[s]);
        }
    }
    *n_near = nn;
    *n_far = nf;
    if (nn > cap_near || nf > cap_far)
        return fail(KRR_ERR_INVALID_ARG, "krr_h_partition: more pairs than the capacities (counts returned)");
    return KRR_OK;
}
