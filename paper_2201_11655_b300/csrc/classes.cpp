// Motif class tables, built once per k on the host.
//
// The motif index of an ordered k-tuple is its adjacency matrix read row by
// row with the diagonal removed, most significant bit first (Definitions,
// Fig. 1: 110101 = 53).  Isomorphic indices are merged into the class named
// by the minimum index (isomorph-merge paragraph of "The Algorithm"; Fig. 1:
// 53 -> 30).
//
// Method used here: orbits.  S_k is generated by the adjacent transpositions
// (i i+1); the class of an index is its orbit under the group, found by a
// closure over those generators, and its name is the smallest member.  Only
// weakly connected orbits (Definitions: a k-motif is connected in G_U) get
// an output column; columns are in ascending order of the class name.
#include <algorithm>
#include <mutex>
#include <vector>

#include "vdmc_internal.cuh"

namespace {

int bit_pos(int k, int i, int j) {
    // position of entry (i, j), i != j, counted from the least significant bit
    int before = i * (k - 1) + (j > i ? j - 1 : j);
    return k * (k - 1) - 1 - before;
}

int entry(int k, int idx, int i, int j) { return (idx >> bit_pos(k, i, j)) & 1; }

// swap vertices t and t+1 of the matrix encoded by idx
int swap_adjacent(int k, int idx, int t) {
    int perm[4] = {0, 1, 2, 3};
    perm[t] = t + 1;
    perm[t + 1] = t;
    int out = 0;
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++)
            if (i != j && entry(k, idx, perm[i], perm[j])) out |= 1 << bit_pos(k, i, j);
    return out;
}

bool weakly_connected(int k, int idx) {
    int parent[4] = {0, 1, 2, 3};
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++)
            if (entry(k, idx, i, j) || entry(k, idx, j, i)) parent[find(i)] = find(j);
    for (int i = 1; i < k; i++)
        if (find(i) != find(0)) return false;
    return true;
}

struct Table {
    std::vector<uint8_t> lut;
    std::vector<uint16_t> canon;
    // undirected variant: the classes whose matrices are symmetric (an
    // orbit of a symmetric matrix holds only symmetric matrices, so its name
    // is the undirected class name); ucol[c] = undirected column of directed
    // column c, 255 if c is not symmetric
    std::vector<uint16_t> ucanon;
    std::vector<uint8_t> ucol;
    // column of each class in the counting kernels' rank-space accumulator
    // (acc_col) and its inverse (acc_class); see accumulator_order
    std::vector<uint8_t> acc_col, acc_class;
};

// 12-bit index of the 4-tuple (r, a, b, c) from its six pair flags (Fig. 1
// bit order; the same packing as the kernels' mask4)
int index4(int fra, int frb, int frc, int fab, int fac, int fbc) {
    return ((fra & 1) << 11) | ((frb & 1) << 10) | ((frc & 1) << 9) | ((fra >> 1) << 8) | ((fab & 1) << 7) |
           ((fac & 1) << 6) | ((frb >> 1) << 5) | ((fab >> 1) << 4) | ((fbc & 1) << 3) | ((frc >> 1) << 2) |
           ((fac >> 1) << 1) | (fbc >> 1);
}

// Accumulator column order (k = 4).  The root-per-CTA kernel credits a
// second-hop vertex c of a member v (colour al, h(v, c) = f) in the classes
// of r-v-c with a partner be of r, and of r-v-{c, c2}; and a second-hop
// vertex b with a P-neighbour of type (c1, h1) in the classes of r-x-b-c.
// Those 25 classes come first, each group's new classes next to each other,
// so that the few atomics one (v, c) or b adds land in one or two 128-byte
// lines of the vertex's row; the other classes follow in ascending order.
// Counts do not depend on the order (the un-relabel pass maps it back).
std::vector<uint8_t> accumulator_order(int k, const std::vector<uint8_t> &lut, int nclasses) {
    std::vector<uint8_t> order;
    std::vector<char> used(nclasses, 0);
    auto take = [&](int idx) {
        const int c = lut[idx];
        if (c < nclasses && !used[c]) {
            used[c] = 1;
            order.push_back((uint8_t)c);
        }
    };
    if (k == 4) {
        for (int al = 1; al <= 3; al++)
            for (int f = 1; f <= 3; f++) {
                for (int be = 1; be <= 3; be++) take(index4(al, be, 0, 0, f, 0));
                for (int f2 = 1; f2 <= 3; f2++) take(index4(al, 0, 0, f, f2, 0));
            }
        for (int c1 = 1; c1 <= 3; c1++)
            for (int h1 = 1; h1 <= 3; h1++)
                for (int f = 1; f <= 3; f++) take(index4(c1, 0, 0, h1, 0, f));
    }
    for (int c = 0; c < nclasses; c++)
        if (!used[c]) order.push_back((uint8_t)c);
    return order;
}

bool symmetric(int k, int idx) {
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++)
            if (entry(k, idx, i, j) != entry(k, idx, j, i)) return false;
    return true;
}

Table build(int k) {
    const int nidx = 1 << (k * (k - 1));
    std::vector<int> name(nidx, -1);
    std::vector<int> stack, orbit;
    for (int start = 0; start < nidx; start++) {
        if (name[start] >= 0) continue;
        orbit.clear();
        stack.assign(1, start);
        name[start] = start;
        while (!stack.empty()) {
            int x = stack.back();
            stack.pop_back();
            orbit.push_back(x);
            for (int t = 0; t + 1 < k; t++) {
                int y = swap_adjacent(k, x, t);
                if (name[y] < 0) {
                    name[y] = start;
                    stack.push_back(y);
                }
            }
        }
        int lo = *std::min_element(orbit.begin(), orbit.end());
        for (int x : orbit) name[x] = lo;
    }
    Table T;
    for (int idx = 0; idx < nidx; idx++)
        if (name[idx] == idx && weakly_connected(k, idx)) T.canon.push_back((uint16_t)idx);
    T.lut.assign(nidx, 255);
    for (int idx = 0; idx < nidx; idx++) {
        if (!weakly_connected(k, idx)) continue;
        auto it = std::lower_bound(T.canon.begin(), T.canon.end(), (uint16_t)name[idx]);
        T.lut[idx] = (uint8_t)(it - T.canon.begin());
    }
    T.acc_class = accumulator_order(k, T.lut, (int)T.canon.size());
    T.acc_col.assign(T.canon.size(), 255);
    for (size_t j = 0; j < T.acc_class.size(); j++) T.acc_col[T.acc_class[j]] = (uint8_t)j;
    T.ucol.assign(T.canon.size(), 255);
    for (size_t c = 0; c < T.canon.size(); c++)
        if (symmetric(k, T.canon[c])) {
            T.ucol[c] = (uint8_t)T.ucanon.size();
            T.ucanon.push_back(T.canon[c]);
        }
    return T;
}

Table g_tab[5];
std::once_flag g_once[5];

const Table *table(int k) {
    if (k != 3 && k != 4) return nullptr;
    std::call_once(g_once[k], [k] { g_tab[k] = build(k); });
    return &g_tab[k];
}

}  // namespace

const uint8_t *vdmc_host_lut(int k) {
    const Table *t = table(k);
    return t ? t->lut.data() : nullptr;
}

const uint16_t *vdmc_host_canon(int k, int *num_classes) {
    const Table *t = table(k);
    if (!t) return nullptr;
    if (num_classes) *num_classes = (int)t->canon.size();
    return t->canon.data();
}

const uint8_t *vdmc_host_acc_col(int k) {
    const Table *t = table(k);
    return t ? t->acc_col.data() : nullptr;
}

const uint8_t *vdmc_host_acc_class(int k) {
    const Table *t = table(k);
    return t ? t->acc_class.data() : nullptr;
}

const uint8_t *vdmc_host_ucol(int k, int *num_undirected) {
    const Table *t = table(k);
    if (!t) return nullptr;
    if (num_undirected) *num_undirected = (int)t->ucanon.size();
    return t->ucol.data();
}

extern "C" int vdmc_num_classes_undirected(int k) {
    int nu = -1;
    if (!vdmc_host_ucol(k, &nu)) return -1;
    return nu;
}

extern "C" vdmc_status vdmc_undirected_class_masks(int k, uint16_t *canon_out) {
    const Table *t = table(k);
    if (!t || !canon_out) return VDMC_ERR_INVALID_ARG;
    std::copy(t->ucanon.begin(), t->ucanon.end(), canon_out);
    return VDMC_OK;
}

extern "C" int vdmc_num_classes(int k) {
    int nc = -1;
    if (!vdmc_host_canon(k, &nc)) return -1;
    return nc;
}

extern "C" vdmc_status vdmc_class_masks(int k, uint16_t *canon_out) {
    int nc = 0;
    const uint16_t *c = vdmc_host_canon(k, &nc);
    if (!c || !canon_out) return VDMC_ERR_INVALID_ARG;
    std::copy(c, c + nc, canon_out);
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_class_lut(int k, uint8_t *lut_out) {
    const uint8_t *l = vdmc_host_lut(k);
    if (!l || !lut_out) return VDMC_ERR_INVALID_ARG;
    std::copy(l, l + ((size_t)1 << (k * (k - 1))), lut_out);
    return VDMC_OK;
}
