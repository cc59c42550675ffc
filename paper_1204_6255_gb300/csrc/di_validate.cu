// Consistency check of a graph's arrays (host code; diagnostics, not on the solve path).
//
// di_csr_validate checks the build's invariants on host copies of the arrays: both CSRs are
// well formed (row pointers from 0 to L, non-decreasing; ids in range; each row strictly
// ascending, so sorted and free of duplicates), the degrees are the row lengths, the in-CSR is
// the transpose of the out-CSR (equal order-independent checksums of the link set, and equal
// degree sums), the loop flags mark exactly the rows that hold their own id, and E with its
// levels satisfies its definition (Section 2.4): a node is in E exactly when all of its
// in-neighbours are, and its level is one more than the largest level among them (0 without
// in-neighbours). di_graph_validate copies a built graph's arrays out and checks them, plus the
// push kernels' hub-marked copy of the out-links.
#include <cstring>
#include <vector>

#include "di_internal.cuh"

namespace {

uint64_t mix(uint64_t x) {   // SplitMix64 finaliser (Steele, Lea, Flood): an order-free link hash
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

void check_csr(const char *name, int32_t n, const int64_t *rp, const int32_t *col, int64_t L) {
    DI_REQUIRE(rp[0] == 0 && rp[n] == L, DI_ERR_CORRUPT, "%s: row pointers run from %lld to %lld, not 0 to %lld",
               name, (long long)rp[0], (long long)rp[n], (long long)L);
    for (int32_t i = 0; i < n; i++) {
        DI_REQUIRE(rp[i + 1] >= rp[i] && rp[i + 1] <= L, DI_ERR_CORRUPT,
                   "%s: row pointer decreases or passes L at row %d", name, i);
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            DI_REQUIRE(col[k] >= 0 && col[k] < n, DI_ERR_CORRUPT, "%s: id %d out of range in row %d", name, col[k], i);
            DI_REQUIRE(k == rp[i] || col[k] > col[k - 1], DI_ERR_CORRUPT,
                       "%s: row %d is not strictly ascending at entry %lld", name, i, (long long)(k - rp[i]));
        }
    }
}

}  // namespace

using namespace di;

extern "C" di_status di_csr_validate(int32_t n, int64_t L, const int64_t *rp_out, const int32_t *col_out,
                                     const int64_t *rp_in, const int32_t *col_in, const int32_t *out_deg,
                                     const int32_t *in_deg, const uint8_t *loop, const uint8_t *e_mask,
                                     const int32_t *e_level) {
    return guarded([&] {
        DI_REQUIRE(n >= 1 && L >= 0, DI_ERR_INVALID_ARG, "n = %d, L = %lld", n, (long long)L);
        DI_REQUIRE(rp_out && col_out && rp_in && col_in, DI_ERR_INVALID_ARG, "a CSR array is NULL");
        check_csr("out-CSR", n, rp_out, col_out, L);
        check_csr("in-CSR", n, rp_in, col_in, L);
        uint64_t h_out = 0, h_in = 0;
        for (int32_t i = 0; i < n; i++) {
            for (int64_t k = rp_out[i]; k < rp_out[i + 1]; k++) h_out += mix(((uint64_t)(uint32_t)i << 32) | (uint32_t)col_out[k]);
            for (int64_t k = rp_in[i]; k < rp_in[i + 1]; k++) h_in += mix(((uint64_t)(uint32_t)col_in[k] << 32) | (uint32_t)i);
        }
        DI_REQUIRE(h_out == h_in, DI_ERR_CORRUPT, "the in-CSR is not the transpose of the out-CSR");
        for (int32_t i = 0; i < n; i++) {
            if (out_deg)
                DI_REQUIRE(out_deg[i] == rp_out[i + 1] - rp_out[i], DI_ERR_CORRUPT, "out-degree of node %d", i);
            if (in_deg) DI_REQUIRE(in_deg[i] == rp_in[i + 1] - rp_in[i], DI_ERR_CORRUPT, "in-degree of node %d", i);
            if (loop) {
                bool self = false;
                for (int64_t k = rp_out[i]; k < rp_out[i + 1]; k++) self = self || col_out[k] == i;
                DI_REQUIRE((loop[i] != 0) == self, DI_ERR_CORRUPT, "loop flag of node %d", i);
            }
        }
        if (e_mask && e_level) {
            for (int32_t i = 0; i < n; i++) {
                bool all_in = true;
                int32_t top = -1;
                for (int64_t k = rp_in[i]; k < rp_in[i + 1]; k++) {
                    const int32_t j = col_in[k];
                    all_in = all_in && e_mask[j] != 0;
                    if (e_level[j] > top) top = e_level[j];
                }
                DI_REQUIRE((e_mask[i] != 0) == all_in, DI_ERR_CORRUPT, "E membership of node %d", i);
                DI_REQUIRE(e_mask[i] ? e_level[i] == top + 1 : e_level[i] == -1, DI_ERR_CORRUPT, "E level of node %d",
                           i);
            }
        }
    });
}

extern "C" di_status di_graph_validate(const di_graph *g) {
    return guarded([&] {
        DI_REQUIRE(g != nullptr, DI_ERR_INVALID_ARG, "graph is NULL");
        DeviceGuard dg(g->dev.device);
        const size_t n = (size_t)g->n, L = (size_t)g->L;
        std::vector<int64_t> rp_out(n + 1), rp_in(n + 1);
        std::vector<int32_t> col_out(L + 1), col_in(L + 1), col_push(L + 1), out_deg(n), in_deg(n), e_level(n), hubs(kHubSlots);
        std::vector<uint8_t> loop(n), e_mask(n);
        auto get = [&](void *dst, const DevBuf &b, size_t bytes) {
            if (bytes) DI_CHECK_CUDA(cudaMemcpy(dst, b.p, bytes, cudaMemcpyDeviceToHost));
        };
        get(rp_out.data(), g->rp_out, 8 * (n + 1));
        get(rp_in.data(), g->rp_in, 8 * (n + 1));
        get(col_out.data(), g->col_out, 4 * L);
        get(col_in.data(), g->col_in, 4 * L);
        get(col_push.data(), g->col_push, 4 * L);
        get(out_deg.data(), g->out_deg, 4 * n);
        get(in_deg.data(), g->in_deg, 4 * n);
        get(loop.data(), g->loop, n);
        get(e_mask.data(), g->e_mask, n);
        get(e_level.data(), g->e_level, 4 * n);
        get(hubs.data(), g->hub_ids, 4 * kHubSlots);
        const di_status st = di_csr_validate(g->n, g->L, rp_out.data(), col_out.data(), rp_in.data(), col_in.data(),
                                             out_deg.data(), in_deg.data(), loop.data(), e_mask.data(), e_level.data());
        if (st != DI_OK) throw Fail{st};
        // the push's copy: col_out with bit 31 on links into a hub, and a loop node's self-link
        // swapped with the last link of its row
        auto marked = [&](int32_t j) {
            const int32_t slot = (int32_t)(((uint32_t)j * 0x9E3779B1u) >> 21);
            return hubs[slot] == j ? (int32_t)((uint32_t)j | 0x80000000u) : j;
        };
        for (size_t u = 0; u < n; u++) {
            const int64_t b = rp_out[u], e = rp_out[u + 1];
            int64_t self = -1;
            if (loop[u])
                for (int64_t k = b; k < e; k++)
                    if (col_out[k] == (int32_t)u) self = k;
            for (int64_t k = b; k < e; k++) {
                const int64_t src = self < 0 ? k : (k == self ? e - 1 : (k == e - 1 ? self : k));
                DI_REQUIRE(col_push[k] == marked(col_out[src]), DI_ERR_CORRUPT,
                           "the push's link copy differs at link %lld", (long long)k);
            }
        }
        int64_t e_count = 0;
        for (size_t i = 0; i < n; i++) e_count += e_mask[i] != 0;
        DI_REQUIRE(e_count == g->stats.E, DI_ERR_CORRUPT, "|E| = %lld but the statistics say %lld", (long long)e_count,
                   (long long)g->stats.E);
    });
}
