// Mesh extraction of one object (section 4's object meshes, queried inside
// the object's 3D bound): occupancy on a (res+1)^3 lattice over c +- half
// (the query mode of the tile kernel), then marching tetrahedra. Each cube
// splits into the six Kuhn tetrahedra [0, e_a, e_a + e_b, 7] for
// (a, b) = (0,1), (0,2), (1,0), (1,2), (2,0), (2,1) (corner id x + 2y + 4z),
// so neighbouring cubes split shared faces alike and the surface is closed.
// A lattice vertex is inside when its occupancy exceeds the level. Per
// tetrahedron: one vertex alone on its side at position a, others b < c < d:
// triangle (E(a,b), E(a,c), E(a,d)); two inside i < j and two outside k < l:
// (E(i,k), E(i,l), E(j,l)) and (E(i,k), E(j,l), E(j,k)). E interpolates the
// level crossing from the lower tetrahedron position to the higher one; each
// triangle is turned so (B - A) x (C - A) points from the inside vertices'
// centroid to the outside ones'. Triangles are written in cube order (x
// fastest), tetrahedron order, then the order above: a count pass, a scan
// and an emit pass make the output deterministic.
#pragma once
#include "vmap_build.cuh"
#include "vmap_common.cuh"

namespace vmapk {

struct MtGrid {
    const float* occ;     // [(res+1)^3], vertex i + (res+1)(j + (res+1) k)
    int res;
    float o[3], s[3];     // lattice origin (c - half) and spacing (2 half / res)
    float level;
};

__global__ void k_lattice_points(float* pts, int res, float ox, float oy, float oz, float sx, float sy, float sz) {
    const long long n1 = res + 1, nv = n1 * n1 * n1;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % n1), j = (int)((v / n1) % n1), k = (int)(v / (n1 * n1));
        pts[3 * v] = ox + (float)i * sx;
        pts[3 * v + 1] = oy + (float)j * sy;
        pts[3 * v + 2] = oz + (float)k * sz;
    }
}

__device__ __forceinline__ void mt_edge(const float (&P)[4][3], const float (&F)[4], int x, int y, float level,
                                        float (&e)[3]) {
    const int lo = min(x, y), hi = max(x, y);
    const float t = (level - F[lo]) / (F[hi] - F[lo]);
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] = P[lo][a] + t * (P[hi][a] - P[lo][a]);
}

// write triangle (A, B, C), turned to face from the inside centroid to the outside one
__device__ __forceinline__ void mt_put(float* out, const float (&A)[3], const float (&B)[3], const float (&C)[3],
                                       const float (&g)[3]) {
    const float u0 = B[0] - A[0], u1 = B[1] - A[1], u2 = B[2] - A[2];
    const float v0 = C[0] - A[0], v1 = C[1] - A[1], v2 = C[2] - A[2];
    const float n0 = u1 * v2 - u2 * v1, n1 = u2 * v0 - u0 * v2, n2 = u0 * v1 - u1 * v0;
    const bool flip = n0 * g[0] + n1 * g[1] + n2 * g[2] < 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out[a] = A[a];
        out[3 + a] = flip ? C[a] : B[a];
        out[6 + a] = flip ? B[a] : C[a];
    }
}

// triangles of one tetrahedron; writes them to out (9 floats each) when out != NULL
__device__ __forceinline__ int mt_tet(const float (&P)[4][3], const float (&F)[4], float level, float* out) {
    int in = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) in |= (F[q] > level ? 1 : 0) << q;
    const int cnt = __popc(in);
    if (cnt == 0 || cnt == 4) return 0;
    if (!out) return cnt == 2 ? 2 : 1;
    float g[3], pin[3] = {0.f, 0.f, 0.f}, pout[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if ((in >> q) & 1) pin[a] += P[q][a];
            else pout[a] += P[q][a];
        }
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] = pout[a] / (float)(4 - cnt) - pin[a] / (float)cnt;
    if (cnt != 2) {
        const int lone_side = cnt == 1 ? 1 : 0;
        int lone = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (((in >> q) & 1) == lone_side) lone = q;
        int r[3], nr = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q != lone) r[nr++] = q;
        float A[3], B[3], C[3];
        mt_edge(P, F, lone, r[0], level, A);
        mt_edge(P, F, lone, r[1], level, B);
        mt_edge(P, F, lone, r[2], level, C);
        mt_put(out, A, B, C, g);
        return 1;
    }
    int ins[2], outs[2], ni = 0, no = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if ((in >> q) & 1) ins[ni++] = q;
        else outs[no++] = q;
    }
    float eik[3], eil[3], ejl[3], ejk[3];
    mt_edge(P, F, ins[0], outs[0], level, eik);
    mt_edge(P, F, ins[0], outs[1], level, eil);
    mt_edge(P, F, ins[1], outs[1], level, ejl);
    mt_edge(P, F, ins[1], outs[0], level, ejk);
    mt_put(out, eik, eil, ejl, g);
    mt_put(out + 9, eik, ejl, ejk, g);
    return 2;
}

// triangles of cube q (all six tetrahedra); writes them when out != NULL
__device__ int mt_cube(const MtGrid& g, long long q, float* out) {
    const int res = g.res;
    const long long n1 = res + 1;
    const int i = (int)(q % res), j = (int)((q / res) % res), k = (int)(q / ((long long)res * res));
    float cf[8], cp[8][3];
    bool any_in = false, any_out = false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int vi = i + (c & 1), vj = j + ((c >> 1) & 1), vk = k + ((c >> 2) & 1);
        cf[c] = g.occ[vi + n1 * (vj + n1 * vk)];
        cp[c][0] = g.o[0] + (float)vi * g.s[0];
        cp[c][1] = g.o[1] + (float)vj * g.s[1];
        cp[c][2] = g.o[2] + (float)vk * g.s[2];
        if (cf[c] > g.level) any_in = true;
        else any_out = true;
    }
    if (!(any_in && any_out)) return 0;
    const int ka[6] = {0, 0, 1, 1, 2, 2}, kb[6] = {1, 2, 0, 2, 0, 1};
    int n = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        const int cid[4] = {0, 1 << ka[t], (1 << ka[t]) | (1 << kb[t]), 7};
        float P[4][3], F[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            F[v] = cf[cid[v]];
#pragma unroll
            for (int a = 0; a < 3; ++a) P[v][a] = cp[cid[v]][a];
        }
        n += mt_tet(P, F, g.level, out ? out + 9 * n : nullptr);
    }
    return n;
}

__global__ void k_mt_count(MtGrid g, int* counts) {
    const long long nc = (long long)g.res * g.res * g.res;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nc; q += (long long)gridDim.x * blockDim.x)
        counts[q] = mt_cube(g, q, nullptr);
}

// exclusive scan of n counts into offs[0..n] (offs[n] = total), one block of BUILD_THREADS
__global__ void __launch_bounds__(BUILD_THREADS) k_scan_counts(const int* counts, long long n, long long* offs) {
    __shared__ long long sh[64];
    const long long per = (n + BUILD_THREADS - 1) / BUILD_THREADS;
    const long long b = threadIdx.x * per, e = min(n, b + per);
    long long local = 0;
    for (long long q = b; q < e; ++q) local += counts[q];
    long long total;
    long long run = block_scan(local, &total, sh);
    for (long long q = b; q < e; ++q) {
        offs[q] = run;
        run += counts[q];
    }
    if (threadIdx.x == 0) offs[n] = total;
}

__global__ void k_mt_emit(MtGrid g, const long long* offs, float* tris, long long max_tris) {
    const long long nc = (long long)g.res * g.res * g.res;
    float buf[12 * 9];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nc; q += (long long)gridDim.x * blockDim.x) {
        const long long o = offs[q];
        if (offs[q + 1] == o) continue;
        const int n = mt_cube(g, q, buf);
        for (int t = 0; t < n && o + t < max_tris; ++t)
            for (int a = 0; a < 9; ++a) tris[(o + t) * 9 + a] = buf[9 * t + a];
    }
}

}  // namespace vmapk
