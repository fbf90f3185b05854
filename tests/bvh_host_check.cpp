// Host-side driver for the CPU tests of the BVH builder's FP16 node packing (bvh.cpp):
// reads its input from a binary file, writes what the library computed to another, so
// that the Python test checks it against numpy's own binary16 decoding.
//   half  <in: float32[n]>            <out: uint16[n][2] = (rounded down, rounded up)>
//   pack  <in: int32 n, float32[n][9]> <out: int64 nodes, BvhNode[nodes], int32 ok,
//                                       BvhNodeH[nodes]>
//   limit <unused>                    <out: int32[3] = pack results for a leaf of 31
//                                       references, of 32, and a first reference 2^26>
//   growth <in: as pack>              <out: float64 mean surface-area growth of the
//                                       packed child boxes>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "bvh.h"

using namespace nrrs;

static std::vector<char> slurp(const char* path) {
    std::vector<char> b;
    FILE* f = std::fopen(path, "rb");
    if (!f) return b;
    char buf[65536];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) b.insert(b.end(), buf, buf + k);
    std::fclose(f);
    return b;
}

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    const std::vector<char> in = slurp(argv[2]);
    FILE* out = std::fopen(argv[3], "wb");
    if (!out) return 2;
    if (!std::strcmp(argv[1], "half")) {
        const size_t n = in.size() / 4;
        for (size_t i = 0; i < n; ++i) {
            float x;
            std::memcpy(&x, in.data() + 4 * i, 4);
            const uint16_t r[2] = {half_directed(x, false), half_directed(x, true)};
            std::fwrite(r, 2, 2, out);
        }
    } else if (!std::strcmp(argv[1], "pack") || !std::strcmp(argv[1], "growth")) {
        int32_t n;
        std::memcpy(&n, in.data(), 4);
        std::vector<float> tri((size_t)n * 9);
        std::memcpy(tri.data(), in.data() + 4, tri.size() * 4);
        std::vector<int32_t> mat((size_t)n, 0);
        BvhHost b;
        build_bvh(tri.data(), n, mat.data(), &b);
        std::vector<BvhNodeH> h;
        const int32_t ok = pack_half_nodes(b, &h) ? 1 : 0;
        if (!std::strcmp(argv[1], "growth")) {
            const double g = half_node_growth(b, h);
            std::fwrite(&g, 8, 1, out);
            std::fclose(out);
            return 0;
        }
        const int64_t nn = (int64_t)b.nodes.size();
        std::fwrite(&nn, 8, 1, out);
        std::fwrite(b.nodes.data(), sizeof(BvhNode), b.nodes.size(), out);
        std::fwrite(&ok, 4, 1, out);
        std::fwrite(h.data(), sizeof(BvhNodeH), h.size(), out);
    } else if (!std::strcmp(argv[1], "limit")) {
        // one root with a leaf child of (first, count)
        const int32_t cases[3][2] = {{0, 31}, {0, 32}, {1 << 26, 1}};
        for (const auto& c : cases) {
            BvhHost b;
            b.nodes.resize(1);
            BvhNode& r = b.nodes[0];
            for (int k = 0; k < 4; ++k) r.a[k] = r.b[k] = r.c[k] = 0.0f;
            r.d[0] = ~c[0];
            r.d[1] = ~0;
            r.d[2] = c[1];
            r.d[3] = 0;
            std::vector<BvhNodeH> h;
            const int32_t ok = pack_half_nodes(b, &h) ? 1 : 0;
            std::fwrite(&ok, 4, 1, out);
        }
    } else {
        std::fclose(out);
        return 2;
    }
    std::fclose(out);
    return 0;
}
