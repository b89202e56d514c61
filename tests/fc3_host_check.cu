// Host-side check of the 3D octree code of libfc (Morton order, hash index,
// regrid with 2:1 balance, neighbour tables), no GPU needed: reads leaves,
// flags and the level range, regrids, checks every table entry for
// consistency with the forest and prints the new leaves.
//
//   fc3_host_check <in> <out>     in: "n lmin lmax" then n lines "level x y z flag"
#include "../paper_1308_1472_gb300/csrc/fc3_api.cu"

#include <cstdio>

static int fail(const char *what, int i, int t)
{
    std::printf("FAIL %s leaf %d direction %d\n", what, i, t);
    return 1;
}

int main(int argc, char **argv)
{
    if (argc != 3) return 2;
    FILE *f = std::fopen(argv[1], "r");
    int n, lmin, lmax;
    if (!f || std::fscanf(f, "%d %d %d", &n, &lmin, &lmax) != 3) return 2;
    fc3::Forest3 F;
    std::vector<int8_t> flags(n);
    for (int i = 0; i < n; ++i) {
        int l, x, y, z, fl;
        if (std::fscanf(f, "%d %d %d %d %d", &l, &x, &y, &z, &fl) != 5) return 2;
        F.L.push_back(fc3::Leaf3{fc3::key3(l, x, y, z), l, x, y, z});
        flags[i] = (int8_t)fl;
    }
    std::fclose(f);
    F.index();
    if (!F.covers() || !F.balanced()) { std::printf("FAIL input forest\n"); return 1; }
    fc3::Forest3 G;
    if (fc3::regrid_forest(F, flags.data(), lmin, lmax, G)) { std::printf("FAIL regrid %s\n", fc_last_error()); return 1; }
    if (!G.covers() || !G.balanced()) { std::printf("FAIL regridded forest\n"); return 1; }
    fc3::Tables T;
    if (fc3::build_tables(G, T)) { std::printf("FAIL tables %s\n", fc_last_error()); return 1; }
    // every table entry against the forest
    int bad = 0;
    for (int i = 0; i < G.n(); ++i) {
        const fc3::Leaf3 &q = G.L[i];
        const int w = 1 << q.l;
        int t = 0;
        for (int d = 0; d < 27; ++d) {
            if (d == 13) continue;
            const int dir[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
            const int b[3] = {fc3::wrapi(q.x + dir[0], w), fc3::wrapi(q.y + dir[1], w), fc3::wrapi(q.z + dir[2], w)};
            const int *en = &T.nb[((size_t)i * 26 + t) * 5];
            if (en[0] == 1) {
                const fc3::Leaf3 &r = G.L[en[1]];
                if (r.l != q.l || r.x != b[0] || r.y != b[1] || r.z != b[2]) bad |= fail("same-level entry", i, t);
            } else if (en[0] == 2) {
                const fc3::Leaf3 &r = G.L[en[1]];
                if (r.l != q.l - 1 || r.x != b[0] >> 1 || r.y != b[1] >> 1 || r.z != b[2] >> 1) bad |= fail("coarser entry", i, t);
                if (T.tslot[en[1]] < 0) bad |= fail("coarser leaf without a tile", i, t);
            } else if (en[0] == 3) {
                int nf = 0, fa[3];
                for (int a = 0; a < 3; ++a) if (dir[a] == 0) fa[nf++] = a;
                for (int s = 0; s < (1 << nf); ++s) {
                    int c[3];
                    for (int a = 0; a < 3; ++a) c[a] = 2 * b[a] + (dir[a] > 0 ? 0 : 1);
                    for (int k = 0; k < nf; ++k) c[fa[k]] = 2 * b[fa[k]] + ((s >> k) & 1);
                    const fc3::Leaf3 &r = G.L[en[1 + s]];
                    if (r.l != q.l + 1 || r.x != c[0] || r.y != c[1] || r.z != c[2]) bad |= fail("finer entry", i, t);
                }
                if (T.tslot[i] < 0) bad |= fail("leaf beside a finer one without a tile", i, t);
                if (std::abs(dir[0]) + std::abs(dir[1]) + std::abs(dir[2]) == 1 && T.fslot[i] < 0)
                    bad |= fail("face beside finer leaves without records", i, t);
            } else {
                bad |= fail("entry kind", i, t);
            }
            ++t;
        }
    }
    FILE *o = std::fopen(argv[2], "w");
    for (const fc3::Leaf3 &q : G.L) std::fprintf(o, "%d %d %d %d\n", q.l, q.x, q.y, q.z);
    std::fclose(o);
    std::printf(bad ? "FAIL\n" : "ok %d\n", G.n());
    return bad;
}
