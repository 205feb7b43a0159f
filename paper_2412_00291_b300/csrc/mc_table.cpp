// Marching-cubes case table and class palette, generated at load time.
//
// The table is derived here from one rule rather than copied from any
// published table.  For a cube whose corners are classified inside (D < 0)
// or outside, each face contributes directed segments: walking the face's
// corners counter-clockwise about its outward normal, an edge going from an
// outside to an inside corner ("entering") is joined to the next edge going
// from inside to outside ("leaving").  On a face with four crossings this
// separates the two inside corners.  Every crossing cube edge is entering
// on one of its two faces and leaving on the other, so the segments close
// into loops; each loop is fanned from the vertex whose lattice edge has the
// smallest key (lower end offset (dz, dy, dx), then axis), which orients the
// triangles toward positive distance.
//
// Corner c = dx + 2 dy + 4 dz.  Cube edge e = axis * 4 + d1 + 2 d2, running
// along `axis` from the corner with offset d1 on axis (axis+1)%3 and d2 on
// axis (axis+2)%3.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/semtsdf.h"

namespace {

// faces as corner ids, counter-clockwise seen from outside the cube
const int kFaces[6][4] = {
    {0, 4, 6, 2},   // x = 0
    {1, 3, 7, 5},   // x = 1
    {0, 1, 5, 4},   // y = 0
    {2, 6, 7, 3},   // y = 1
    {0, 2, 3, 1},   // z = 0
    {4, 5, 7, 6},   // z = 1
};

int bit(int c, int axis) { return (c >> axis) & 1; }

int cube_edge(int ca, int cb) {
    const int diff = ca ^ cb;
    const int axis = diff == 1 ? 0 : (diff == 2 ? 1 : 2);
    const int lo = ca < cb ? ca : cb;
    return axis * 4 + bit(lo, (axis + 1) % 3) + 2 * bit(lo, (axis + 2) % 3);
}

int edge_rank(int e) {
    const int axis = e >> 2, d1 = e & 1, d2 = (e >> 1) & 1;
    int off[3] = {0, 0, 0};
    off[(axis + 1) % 3] = d1;
    off[(axis + 2) % 3] = d2;
    return ((off[2] * 2 + off[1]) * 2 + off[0]) * 3 + axis;
}

struct Tables {
    int8_t tri[256][MAP_MC_MAXTRI][3];
    int ok = 0;
    Tables() {
        std::memset(tri, -1, sizeof(tri));
        // every face listing must wind counter-clockwise about its outward normal
        for (int f = 0; f < 6; ++f) {
            double P[4][3];
            for (int j = 0; j < 4; ++j)
                for (int k = 0; k < 3; ++k) P[j][k] = bit(kFaces[f][j], k);
            double a[3], b[3], n[3];
            for (int k = 0; k < 3; ++k) {
                a[k] = P[1][k] - P[0][k];
                b[k] = P[2][k] - P[1][k];
            }
            n[0] = a[1] * b[2] - a[2] * b[1];
            n[1] = a[2] * b[0] - a[0] * b[2];
            n[2] = a[0] * b[1] - a[1] * b[0];
            const int axis = f / 2;
            const double want = (f % 2) ? 1.0 : -1.0;
            if (n[axis] != want) return;
        }
        for (int cs = 0; cs < 256; ++cs) {
            int next[12];
            for (int e = 0; e < 12; ++e) next[e] = -1;
            for (int f = 0; f < 6; ++f)
                for (int j = 0; j < 4; ++j) {
                    const int ca = kFaces[f][j], cb = kFaces[f][(j + 1) & 3];
                    const bool ina = (cs >> ca) & 1, inb = (cs >> cb) & 1;
                    if (ina || !inb) continue;          // want outside -> inside
                    for (int s = 1; s < 4; ++s) {
                        const int cc = kFaces[f][(j + s) & 3], cd = kFaces[f][(j + s + 1) & 3];
                        if (((cs >> cc) & 1) && !((cs >> cd) & 1)) {
                            next[cube_edge(ca, cb)] = cube_edge(cc, cd);
                            break;
                        }
                    }
                }
            bool used[12] = {false};
            int nt = 0;
            for (int e0 = 0; e0 < 12; ++e0) {
                if (next[e0] < 0 || used[e0]) continue;
                std::vector<int> loop;
                for (int e = e0; !used[e]; e = next[e]) {
                    used[e] = true;
                    loop.push_back(e);
                    if (next[e] < 0) return;             // open chain: rule violated
                }
                size_t start = 0;
                for (size_t i = 1; i < loop.size(); ++i)
                    if (edge_rank(loop[i]) < edge_rank(loop[start])) start = i;
                const size_t L = loop.size();
                for (size_t i = 1; i + 1 < L; ++i) {
                    if (nt >= MAP_MC_MAXTRI) return;
                    tri[cs][nt][0] = (int8_t)loop[start];
                    tri[cs][nt][1] = (int8_t)loop[(start + i) % L];
                    tri[cs][nt][2] = (int8_t)loop[(start + i + 1) % L];
                    ++nt;
                }
            }
        }
        ok = 1;
    }
};

const Tables &tables() {
    static const Tables t;
    return t;
}

}  // namespace

extern "C" int32_t map_mc_table(int8_t *table_out) {
    const Tables &t = tables();
    if (!t.ok) return -1;
    if (table_out) std::memcpy(table_out, t.tri, sizeof(t.tri));
    return 0;
}

// Class colours: hue l / C of a full turn at full saturation and value.
extern "C" int32_t map_palette(int32_t n_classes, uint8_t *rgb_out) {
    if (n_classes <= 0 || !rgb_out) return -1;
    for (int l = 0; l < n_classes; ++l) {
        const double h6 = 6.0 * l / n_classes;
        const int i = (int)std::floor(h6) % 6;
        const double f = h6 - std::floor(h6);
        // rising and falling ramps of the hexcone
        const double up = f, down = 1.0 - f;
        double rgb[3];
        const double tab[6][3] = {{1, up, 0}, {down, 1, 0}, {0, 1, up}, {0, down, 1}, {up, 0, 1}, {1, 0, down}};
        for (int k = 0; k < 3; ++k) rgb[k] = tab[i][k];
        for (int k = 0; k < 3; ++k) rgb_out[3 * l + k] = (uint8_t)std::lround(255.0 * rgb[k]);
    }
    return 0;
}
