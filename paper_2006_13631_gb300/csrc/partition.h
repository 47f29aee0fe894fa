// Node order for the FV tiles: recursive bisection of the mesh graph.
// Host-only C++.
#pragma once
#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

namespace hk {

// Splits the nodes 0 .. n-1 of the triangle mesh (tri: nt x 3 node indices)
// into `parts` parts of equal size (+-1) that are compact in graph distance,
// and returns them as one order (order[p] = node) with part k at positions
// part_start[k] .. part_start[k+1]-1.  Recursive bisection: a node set
// meant for q parts is split in the proportion floor(q/2) : q - floor(q/2)
// by the key d_p(v) - d_q(v), the BFS distances (inside the set) from a
// node p far from an arbitrary one and from the node q farthest from p, so
// the cut runs across the set's longest extent in the graph; nodes the BFS
// does not reach go last.  Ties, and the order inside a part, follow mkey
// (the Morton key of the position), then the node index.
inline void partition_order(int n, const int32_t* tri, int nt, const uint64_t* mkey, int parts,
                            std::vector<int32_t>& order, std::vector<int32_t>& part_start) {
    // node adjacency from the triangles
    std::vector<int32_t> aptr(n + 1, 0), adj;
    {
        std::vector<std::vector<int32_t>> nb(n);
        for (int k = 0; k < nt; ++k)
            for (int j = 0; j < 3; ++j) {
                const int a0 = tri[3 * k + j];
                nb[a0].push_back(tri[3 * k + (j + 1) % 3]);
                nb[a0].push_back(tri[3 * k + (j + 2) % 3]);
            }
        for (int i = 0; i < n; ++i) {
            std::sort(nb[i].begin(), nb[i].end());
            nb[i].erase(std::unique(nb[i].begin(), nb[i].end()), nb[i].end());
            adj.insert(adj.end(), nb[i].begin(), nb[i].end());
            aptr[i + 1] = (int32_t)adj.size();
        }
    }
    constexpr int64_t kFar = (int64_t)1 << 40;
    std::vector<int32_t> in_set(n, 0), queue(n);
    std::vector<int64_t> d1(n), d2(n);
    int stamp = 0;
    // BFS within the current set from src; returns the last node reached
    auto bfs = [&](int src, std::vector<int64_t>& dist, const std::vector<int32_t>& S) {
        for (int32_t v : S) dist[v] = kFar;
        dist[src] = 0;
        int qh = 0, qt = 0, last = src;
        queue[qt++] = src;
        while (qh < qt) {
            const int u = queue[qh++];
            last = u;
            for (int e = aptr[u]; e < aptr[u + 1]; ++e) {
                const int v = adj[e];
                if (in_set[v] == stamp && dist[v] == kFar) {
                    dist[v] = dist[u] + 1;
                    queue[qt++] = v;
                }
            }
        }
        return last;
    };
    order.clear();
    order.reserve(n);
    part_start.assign(1, 0);
    struct Job {
        std::vector<int32_t> S;
        int parts;
    };
    std::vector<Job> stack;
    {
        Job j0;
        j0.S.resize(n);
        for (int i = 0; i < n; ++i) j0.S[i] = i;
        j0.parts = parts;
        stack.push_back(std::move(j0));
    }
    while (!stack.empty()) {
        Job job = std::move(stack.back());
        stack.pop_back();
        std::vector<int32_t>& S = job.S;
        if (job.parts <= 1 || S.size() <= 1) {
            std::sort(S.begin(), S.end(), [&](int32_t a0, int32_t b0) {
                return mkey[a0] != mkey[b0] ? mkey[a0] < mkey[b0] : a0 < b0;
            });
            order.insert(order.end(), S.begin(), S.end());
            part_start.push_back((int32_t)order.size());
            continue;
        }
        ++stamp;
        for (int32_t v : S) in_set[v] = stamp;
        const int p0 = bfs(S[0], d1, S);
        const int q0 = bfs(p0, d1, S);
        bfs(q0, d2, S);
        auto key = [&](int32_t v) { return (d1[v] >= kFar || d2[v] >= kFar) ? kFar : d1[v] - d2[v]; };
        std::sort(S.begin(), S.end(), [&](int32_t a0, int32_t b0) {
            const int64_t ka = key(a0), kb = key(b0);
            if (ka != kb) return ka < kb;
            return mkey[a0] != mkey[b0] ? mkey[a0] < mkey[b0] : a0 < b0;
        });
        const int p1 = job.parts / 2;
        const size_t half = S.size() * (size_t)p1 / (size_t)job.parts;
        Job lo, hi;
        lo.S.assign(S.begin(), S.begin() + half);
        lo.parts = p1;
        hi.S.assign(S.begin() + half, S.end());
        hi.parts = job.parts - p1;
        stack.push_back(std::move(hi));  // the first half is taken next
        stack.push_back(std::move(lo));
    }
}

}  // namespace hk
