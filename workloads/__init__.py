"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module only builds inputs -- surface meshes, exterior heat sources and
the workload recipes -- and holds none of the method's arithmetic.

Meshes are closed, conforming triangulations with counter-clockwise vertex
order seen from outside (outward normals), as the space-time tensor-product
mesh of Sec. 3 needs:

* ``cube_mesh(n)``: surface of [lo, hi]^3, n x n squares per face, every
  square split by its diagonal from local (0,0) to (1,1) into two congruent
  triangles (12 n^2 triangles, 6 n^2 + 2 nodes).  The paper's experiments use
  such cube meshes (Sec. 6: 192 ... 12288 triangles).
* ``icosphere(nf, radius)``: class-I geodesic sphere of frequency nf, each
  icosahedron face split into nf^2 triangles, vertices pushed to the sphere
  (20 nf^2 triangles, 10 nf^2 + 2 nodes).
* ``ellipsoid(nf, axes)``: the icosphere scaled along x, y, z.

Sources are arrays [nrhs, n_src, 5] of (y1, y2, y3, t0, weight): the
Dirichlet datum of right-hand side r is sum_s weight_s G_alpha(x - y_s, t - t0_s)
with every y_s outside the domain (the exact-solution setting of Sec. 6.1).
"""
import itertools

import numpy as np


def cube_mesh(n, lo=0.0, hi=1.0, diagonal="main"):
    """Surface of the cube [lo, hi]^3, n x n squares per face, each split in
    two triangles along the diagonal from local (0,0) to (1,1) ("main"), from
    (1,0) to (0,1) ("anti"), or alternating between the two in a checkerboard
    ("alternating"); counter-clockwise seen from outside."""
    if n < 1:
        raise ValueError("n must be >= 1")
    if diagonal not in ("main", "anti", "alternating"):
        raise ValueError("diagonal must be main, anti or alternating")
    h = (hi - lo) / n
    index = {}
    nodes = []

    def node(ijk):
        key = tuple(int(v) for v in ijk)
        if key not in index:
            index[key] = len(nodes)
            nodes.append([lo + h * key[0], lo + h * key[1], lo + h * key[2]])
        return index[key]

    tris = []
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        for side in (0, 1):
            # tangent order (b, c) gives normal +e_a, (c, b) gives -e_a
            t1, t2 = (b, c) if side == 1 else (c, b)
            for i in range(n):
                for k in range(n):
                    def corner(di, dk):
                        p = [0, 0, 0]
                        p[a] = side * n
                        p[t1] = i + di
                        p[t2] = k + dk
                        return node(p)
                    p00, p10, p11, p01 = corner(0, 0), corner(1, 0), corner(1, 1), corner(0, 1)
                    if diagonal == "main" or (diagonal == "alternating" and (i + k) % 2 == 0):
                        tris.append([p00, p10, p11])
                        tris.append([p00, p11, p01])
                    else:
                        tris.append([p00, p10, p01])
                        tris.append([p10, p11, p01])
    return np.asarray(nodes, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def _icosahedron():
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    verts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            verts += [(0.0, s1, s2 * phi), (s1, s2 * phi, 0.0), (s2 * phi, 0.0, s1)]
    verts = np.asarray(verts)
    faces = []
    for i, j, k in itertools.combinations(range(12), 3):
        dij = np.linalg.norm(verts[i] - verts[j])
        djk = np.linalg.norm(verts[j] - verts[k])
        dik = np.linalg.norm(verts[i] - verts[k])
        if max(abs(dij - 2.0), abs(djk - 2.0), abs(dik - 2.0)) < 1e-9:
            faces.append((i, j, k))
    assert len(faces) == 20
    return verts, faces


def icosphere(nf, radius=1.0, center=(0.0, 0.0, 0.0)):
    if nf < 1:
        raise ValueError("frequency must be >= 1")
    verts, faces = _icosahedron()
    index = {}
    nodes = []

    def node(weights):
        # exact key: the (corner, weight) pairs with nonzero weight
        key = tuple(sorted((v, w) for v, w in weights if w != 0))
        if key not in index:
            p = sum(w * verts[v] for v, w in key) / nf
            index[key] = len(nodes)
            nodes.append(p / np.linalg.norm(p))
        return index[key]

    tris = []
    for (A, B, C) in faces:
        grid = {}
        for i in range(nf + 1):
            for j in range(nf + 1 - i):
                k = nf - i - j
                grid[(i, j)] = node([(A, i), (B, j), (C, k)])
        for i in range(nf):
            for j in range(nf - i):
                tris.append([grid[(i, j)], grid[(i + 1, j)], grid[(i, j + 1)]])
                if i + j < nf - 1:
                    tris.append([grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]])
    nodes = np.asarray(nodes) * radius
    tris = np.asarray(tris, dtype=np.int32)
    # orient every triangle outward (the sphere is star-shaped about 0)
    v0, v1, v2 = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(v1 - v0, v2 - v0), v0 + v1 + v2) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    nodes = nodes + np.asarray(center, dtype=np.float64)
    return np.ascontiguousarray(nodes, dtype=np.float64), np.ascontiguousarray(tris)


def ellipsoid(nf, axes):
    nodes, tris = icosphere(nf)
    return np.ascontiguousarray(nodes * np.asarray(axes, dtype=np.float64)), tris


def random_sources(rng, nrhs, n_src=1, r_lo=1.5, r_hi=3.0, t0=0.0):
    """Exterior sources at radius U[r_lo, r_hi] in a uniformly random
    direction, onset time t0, unit weights."""
    out = np.zeros((nrhs, n_src, 5))
    for r in range(nrhs):
        for s in range(n_src):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            out[r, s, :3] = d * rng.uniform(r_lo, r_hi)
            out[r, s, 3] = t0
            out[r, s, 4] = 1.0
    return out


def point_source(y, t0=0.0, weight=1.0):
    return np.asarray([[[y[0], y[1], y[2], t0, weight]]], dtype=np.float64)


# ---- workload recipes --------------------------------------------------------
#
# Quadrature orders default to q_reg = 3 (3x3 conical rule per triangle, 81
# points per separated pair), m_ss = 4 (4^4 Gauss points per sub-domain of
# the regularised rules), projection with a 8x8 conical rule and 16 time points.

def reprsc_points(n_steps=32, T=1.0, n_side=33):
    """Evaluation points of the potential benchmark (Sec. 6.2, Table reprsc:
    1089 x 32 = 34848 space-time points): an n_side x n_side grid on the
    plane x3 = 0 over [-0.5, 0.5]^2, at the midpoint (k + 1/2) h of every
    step.  Returns [n_side^2 * n_steps, 4] = (x1, x2, x3, t), time-major."""
    g = np.linspace(-0.5, 0.5, n_side)
    X, Y = np.meshgrid(g, g, indexing="ij")
    xy = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    h = T / n_steps
    return np.concatenate([np.concatenate([xy, np.full((len(xy), 1), (k + 0.5) * h)], axis=1)
                           for k in range(n_steps)])


def workload(name, alpha=None):
    """Returns dict(nodes, tris, alpha, T, n_steps, sources, name)."""
    if name == "cube192_e16":
        nodes, tris = cube_mesh(4)
        return dict(name=name, nodes=nodes, tris=tris, alpha=1.0 if alpha is None else alpha,
                    T=1.0, n_steps=16, sources=point_source((1.5, 1.5, 1.5), t0=-0.1))
    if name.startswith("cube3072_e"):
        # cube3072_e64 is the full-size workload; cube3072_e8 / _e16 are the
        # same mesh with fewer steps (profiling captures of one launch)
        n_steps = int(name[len("cube3072_e"):])
        nodes, tris = cube_mesh(16)
        return dict(name=name, nodes=nodes, tris=tris, alpha=1.0 if alpha is None else alpha,
                    T=1.0, n_steps=n_steps, sources=point_source((1.5, 1.5, 1.5), t0=0.0))
    if name == "sphere5120_e128":
        nodes, tris = icosphere(16)
        return dict(name=name, nodes=nodes, tris=tris, alpha=1.0 if alpha is None else alpha,
                    T=1.0, n_steps=128,
                    sources=random_sources(np.random.default_rng(3), 1))
    if name == "sphere5120_e256":
        nodes, tris = icosphere(16)
        return dict(name=name, nodes=nodes, tris=tris, alpha=1.0 if alpha is None else alpha,
                    T=1.0, n_steps=256,
                    sources=random_sources(np.random.default_rng(5), 8))
    raise KeyError(name)


def batch_workload(seed=0, n_meshes=64):
    """64 independent ellipsoid problems: frequency nf ~ U{4..16}
    (320..5120 triangles), axes ~ U[0.5, 2]^3, E_t ~ U{16..128},
    alpha = 10^U[-1, 1], one exterior source each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_meshes):
        nf = int(rng.integers(4, 17))
        axes = rng.uniform(0.5, 2.0, size=3)
        n_steps = int(rng.integers(16, 129))
        alpha = float(10.0 ** rng.uniform(-1.0, 1.0))
        nodes, tris = ellipsoid(nf, axes)
        src = random_sources(rng, 1, r_lo=2.5, r_hi=4.0)
        out.append(dict(name="ellipsoid%d" % i, nodes=nodes, tris=tris, alpha=alpha,
                        T=1.0, n_steps=n_steps, sources=src))
    return out
