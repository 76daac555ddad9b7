"""Seeded synthetic inputs for the SBR channel-modelling path.

This module is the only code shared by the FP64 oracle and the CUDA path. It
holds geometry and workload descriptions (triangles, surface ids, materials,
antenna positions, frequency grids) and none of the method's arithmetic: no
ray launching, tracing, reflection, field or channel computation lives here.

A scene is a plain dict of numpy arrays:

    tri          float32 [T, 3, 3]   triangle vertices (metres)
    surface_id   int32   [T]         id of the planar surface a triangle belongs to
    materials    float64 [S, 3]      per surface: eps_r, conductivity (S/m), roughness (m)
    tx           float64 [3]         Tx reference point (array centroid)
    rx           float64 [n_rx, 3]   Rx reference points
    rx_valid     bool    [n_rx]      False for receivers placed inside a building
    freqs        float64 [F]         Hz
    gamma_db_km  float32 [F]         specific atmospheric attenuation (dB/km), Eq. 9 as an input
    disp_deg_km  float32 [F]         specific atmospheric dispersion (deg/km), Eq. 10 as an input
    tx_elem      float64 [Nt, 3]     Tx array element positions (Eq. 11)
    rx_elem      float64 [Nr, 3]     Rx array element positions (Eq. 12)
    N, K                             geodesic subdivision frequency and max reflections
    pol                              'V' or 'H'

Three synthetic workloads:
config 1 (SISO 28 GHz, ground + one box), config 2 (urban grid at 300 GHz,
1024 receivers) and config 3 (indoor room with furniture, 16x16 UPA to 64-ULA
at 100 GHz, 1024 subcarriers). Every random draw uses
``numpy.random.default_rng(seed)`` in the order documented per generator.
"""
from __future__ import annotations

import numpy as np

C0 = 299792458.0

__all__ = [
    "C0", "config1", "config2", "config3", "two_ray", "corner_reflector",
    "shoebox", "scene_summary", "upa_yz", "ula_y",
]


# ----------------------------------------------------------------------------
# geometry helpers (pure mesh construction)
# ----------------------------------------------------------------------------

def _lattice(lo: float, hi: float, n: int) -> np.ndarray:
    """n+1 lattice coordinates from lo to hi, identical for every face that uses them."""
    k = np.arange(n + 1, dtype=np.float64)
    xs = lo + (hi - lo) * k / n
    xs[0], xs[-1] = lo, hi
    return xs


def _grid_face(axis: int, value: float, ua: np.ndarray, va: np.ndarray,
               u_axis: int, v_axis: int) -> np.ndarray:
    """Triangles of an axis-aligned rectangle split into (len(ua)-1)x(len(va)-1) quads.

    Every quad (i,j)-(i+1,j)-(i+1,j+1)-(i,j+1) becomes two triangles that share
    its (i,j)-(i+1,j+1) diagonal. Returns float64 [2*nu*nv, 3, 3].
    """
    nu, nv = len(ua) - 1, len(va) - 1
    tris = np.empty((2 * nu * nv, 3, 3), dtype=np.float64)
    t = 0
    for i in range(nu):
        for j in range(nv):
            corners = []
            for (a, b) in ((i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)):
                p = [0.0, 0.0, 0.0]
                p[axis] = value
                p[u_axis] = ua[a]
                p[v_axis] = va[b]
                corners.append(p)
            tris[t] = (corners[0], corners[1], corners[2])
            tris[t + 1] = (corners[0], corners[2], corners[3])
            t += 2
    return tris


def _box_faces(lo, hi, n: int, faces=("x-", "x+", "y-", "y+", "z+", "z-")):
    """Faces of an axis-aligned box, each split into n x n quads.

    Returns a list of (face name, float64 [2n^2, 3, 3]) in the order requested.
    All faces index the same per-axis lattices, so shared edges are bit-identical.
    """
    lx, ly, lz = (_lattice(lo[a], hi[a], n) for a in range(3))
    out = []
    for name in faces:
        if name == "x-":
            out.append((name, _grid_face(0, lo[0], ly, lz, 1, 2)))
        elif name == "x+":
            out.append((name, _grid_face(0, hi[0], ly, lz, 1, 2)))
        elif name == "y-":
            out.append((name, _grid_face(1, lo[1], lx, lz, 0, 2)))
        elif name == "y+":
            out.append((name, _grid_face(1, hi[1], lx, lz, 0, 2)))
        elif name == "z-":
            out.append((name, _grid_face(2, lo[2], lx, ly, 0, 1)))
        elif name == "z+":
            out.append((name, _grid_face(2, hi[2], lx, ly, 0, 1)))
        else:
            raise ValueError(name)
    return out


def upa_yz(center, n_y: int, n_z: int, spacing: float) -> np.ndarray:
    """Uniform planar array in the y-z plane. Element p = a*n_y + b sits at
    center + ((b - (n_y-1)/2) * spacing) * y + ((a - (n_z-1)/2) * spacing) * z."""
    c = np.asarray(center, dtype=np.float64)
    pts = np.empty((n_z * n_y, 3), dtype=np.float64)
    for a in range(n_z):
        for b in range(n_y):
            pts[a * n_y + b] = c + np.array([0.0, (b - (n_y - 1) / 2) * spacing,
                                             (a - (n_z - 1) / 2) * spacing])
    return pts


def ula_y(center, n: int, spacing: float) -> np.ndarray:
    """Uniform linear array along y: element q at center + (q - (n-1)/2)*spacing*y."""
    c = np.asarray(center, dtype=np.float64)
    pts = np.tile(c, (n, 1))
    pts[:, 1] += (np.arange(n) - (n - 1) / 2) * spacing
    return pts


def _assemble(groups):
    """groups: list of float64 [t,3,3] arrays, one per surface (surface id = position)."""
    tri = np.concatenate(groups, axis=0).astype(np.float32)
    sid = np.concatenate([np.full(len(g), s, dtype=np.int32) for s, g in enumerate(groups)])
    return tri, sid


def _base(name, tri, sid, materials, tx, rx, freqs, N, K, pol="V", gamma=None,
          disp=None, tx_elem=None, rx_elem=None, rx_valid=None, **extra):
    freqs = np.atleast_1d(np.asarray(freqs, dtype=np.float64))
    F = len(freqs)
    rx = np.atleast_2d(np.asarray(rx, dtype=np.float64))
    tx = np.asarray(tx, dtype=np.float64)
    sc = dict(
        name=name, tri=tri, surface_id=sid,
        materials=np.asarray(materials, dtype=np.float64).reshape(-1, 3),
        tx=tx, rx=rx,
        rx_valid=np.ones(len(rx), dtype=bool) if rx_valid is None else rx_valid,
        freqs=freqs,
        gamma_db_km=np.zeros(F, np.float32) if gamma is None else np.asarray(gamma, np.float32),
        disp_deg_km=np.zeros(F, np.float32) if disp is None else np.asarray(disp, np.float32),
        tx_elem=tx[None, :].copy() if tx_elem is None else tx_elem,
        rx_elem=rx[:1].copy() if rx_elem is None else rx_elem,
        N=int(N), K=int(K), pol=pol,
    )
    sc.update(extra)
    return sc


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------

def config1(N: int = 100, K: int = 3):
    """SISO 28 GHz: ground (2 triangles, x in [-20,80], y in [-30,70], diagonal
    (-20,-30)-(80,70)) plus one 20x10x15 m box at x in [30,50], y in [35,45],
    z in [0,15] (12 triangles). Concrete everywhere: eps_r 5.31, 0.48 S/m,
    smooth. Tx (0,0,10), Rx (60,25,1.5). Surfaces: 0 ground, 1..6 box faces
    (x-, x+, y-, y+, z+, z-). No randomness."""
    ground = np.array([[[-20, -30, 0], [80, -30, 0], [80, 70, 0]],
                       [[-20, -30, 0], [80, 70, 0], [-20, 70, 0]]], dtype=np.float64)
    groups = [ground] + [g for _, g in _box_faces((30, 35, 0), (50, 45, 15), 1)]
    tri, sid = _assemble(groups)
    mats = np.tile([5.31, 0.48, 0.0], (len(groups), 1))
    return _base("config1_siso_28GHz", tri, sid, mats, (0.0, 0.0, 10.0), [(60.0, 25.0, 1.5)],
                 [28e9], N, K)


def config2(N: int = 1000, K: int = 6, nx: int = 8, ny: int = 5, sub: int = 11,
            ground_sub: int = 40, rx_grid: int = 32, seed: int = 2, crossing=None):
    """Urban grid at 300 GHz (seed 2).

    nx x ny cells on a 60 m pitch, cell (i, j) centred at (30+60i, 30+60j). Draw
    order per cell (i outer, j inner): footprint width U(15,40), depth U(15,40),
    height U(10,60). Each building contributes 4 facades and a roof, each split
    into sub x sub quads. Ground: ground_sub x ground_sub quads over
    [-20,500] x [-20,320] at z=0 (scaled with nx, ny). Surfaces: 0 ground, then
    per building b: 1+5b .. 5+5b = x-, x+, y-, y+, roof. After the buildings,
    per surface: material type ~ integers(0,3) from (eps_r, sigma) in
    {(5.31,0.5), (6.27,0.1), (3.0,0.01)}, roughness U(0.05,0.3) mm.
    Tx at the street crossing (60*(nx//2), 60*(ny//2), 25), i.e. (240,120,25);
    rx_grid x rx_grid receivers on a 2 m pitch centred below it at z=1.5 (receivers inside a footprint get
    rx_valid False). F=1 at 300 GHz; gamma = 5 dB/km (synthetic stand-in for the
    line-by-line value of Eq. 9). `crossing` = (i, j) moves the Tx and the
    receiver grid to the street crossing (60 i, 60 j); the buildings stay."""
    rng = np.random.default_rng(seed)
    xmax = -20 + 60 * nx + 40
    ymax = -20 + 60 * ny + 40
    ground = _grid_face(2, 0.0, _lattice(-20.0, float(xmax), ground_sub),
                        _lattice(-20.0, float(ymax), ground_sub), 0, 1)
    groups = [ground]
    footprints = []
    for i in range(nx):
        for j in range(ny):
            wx = rng.uniform(15, 40)
            wy = rng.uniform(15, 40)
            h = rng.uniform(10, 60)
            cx, cy = 30 + 60 * i, 30 + 60 * j
            lo = (cx - wx / 2, cy - wy / 2, 0.0)
            hi = (cx + wx / 2, cy + wy / 2, h)
            footprints.append((lo, hi))
            for _, g in _box_faces(lo, hi, sub, faces=("x-", "x+", "y-", "y+", "z+")):
                groups.append(g)
    S = len(groups)
    types = np.array([[5.31, 0.5], [6.27, 0.1], [3.0, 0.01]])
    mats = np.empty((S, 3))
    for s in range(S):
        k = rng.integers(0, 3)
        mats[s, :2] = types[k]
        mats[s, 2] = rng.uniform(0.05e-3, 0.3e-3)
    tri, sid = _assemble(groups)
    cx0, cy0 = 60.0 * (nx // 2), 60.0 * (ny // 2)   # (240, 120) for the 8 x 5 grid
    if crossing is not None:
        cx0, cy0 = 60.0 * crossing[0], 60.0 * crossing[1]
    tx = (cx0, cy0, 25.0)
    g = (np.arange(rx_grid) - (rx_grid - 1) / 2) * 2.0
    rx = np.array([(cx0 + gx, cy0 + gy, 1.5) for gx in g for gy in g])
    valid = np.ones(len(rx), dtype=bool)
    for (lo, hi) in footprints:
        inside = (rx[:, 0] > lo[0]) & (rx[:, 0] < hi[0]) & (rx[:, 1] > lo[1]) & (rx[:, 1] < hi[1])
        valid &= ~inside
    return _base("config2_urban_300GHz", tri, sid, mats, tx, rx, [300e9], N, K,
                 gamma=[5.0], rx_valid=valid)


def config3(N: int = 632, K: int = 4, n_furniture: int = 46, wall_sub: int = 8,
            box_sub: int = 3, F: int = 1024, ny_tx: int = 16, nz_tx: int = 16,
            n_rx: int = 64, seed: int = 3, rx_spacing: float = None):
    """Indoor massive MIMO at 100 GHz (seed 3).

    Room [0,10]x[0,8]x[0,3]: 6 surfaces (x-, x+, y-, y+, ceiling z+, floor z-),
    each split wall_sub x wall_sub. Furniture: n_furniture boxes on the floor,
    draw order per box: size x U(0.3,1.5), size y U(0.3,1.5), height U(0.4,2.0),
    centre x U(sx/2, 10-sx/2), centre y U(sy/2, 8-sy/2); a draw whose footprint
    grown by 0.5 m contains an element of either array is redrawn. Each box face
    is split box_sub x box_sub (6 faces). Surfaces: 0..5 room, then 6 per box.
    Per surface (after the geometry): material type ~ integers(0,3) from the
    config-2 types, roughness U(0.05,0.3) mm. Tx: ny_tx x nz_tx UPA in the y-z
    plane centred at (0.5,4.0,2.0); Rx: n_rx ULA along y centred at
    (8.5,3.0,1.2); spacing lambda/2 at 100 GHz (the Rx ULA takes rx_spacing
    instead when given: a wide array whose elements see different paths). Frequencies
    f_k = 100 GHz + (k - F/2) * 10 GHz / F. gamma(f) = 0.5 + 0.1*(f-100 GHz)/5 GHz
    dB/km (synthetic stand-in). SNR 0:5:30 dB."""
    rng = np.random.default_rng(seed)
    lam = C0 / 100e9
    d = lam / 2
    tx_c = np.array([0.5, 4.0, 2.0])
    rx_c = np.array([8.5, 3.0, 1.2])
    tx_elem = upa_yz(tx_c, ny_tx, nz_tx, d)
    rx_elem = ula_y(rx_c, n_rx, d if rx_spacing is None else rx_spacing)
    groups = [g for _, g in _box_faces((0, 0, 0), (10, 8, 3), wall_sub,
                                       faces=("x-", "x+", "y-", "y+", "z+", "z-"))]
    elems = np.concatenate([tx_elem, rx_elem])
    placed = 0
    while placed < n_furniture:
        sx = rng.uniform(0.3, 1.5)
        sy = rng.uniform(0.3, 1.5)
        h = rng.uniform(0.4, 2.0)
        cx = rng.uniform(sx / 2, 10 - sx / 2)
        cy = rng.uniform(sy / 2, 8 - sy / 2)
        lo = np.array([cx - sx / 2, cy - sy / 2, 0.0])
        hi = np.array([cx + sx / 2, cy + sy / 2, h])
        near = ((elems[:, 0] > lo[0] - 0.5) & (elems[:, 0] < hi[0] + 0.5)
                & (elems[:, 1] > lo[1] - 0.5) & (elems[:, 1] < hi[1] + 0.5))
        if near.any():
            continue
        for _, g in _box_faces(lo, hi, box_sub):
            groups.append(g)
        placed += 1
    S = len(groups)
    types = np.array([[5.31, 0.5], [6.27, 0.1], [3.0, 0.01]])
    mats = np.empty((S, 3))
    for s in range(S):
        k = rng.integers(0, 3)
        mats[s, :2] = types[k]
        mats[s, 2] = rng.uniform(0.05e-3, 0.3e-3)
    tri, sid = _assemble(groups)
    freqs = 100e9 + (np.arange(F) - F // 2) * (10e9 / F)
    gamma = 0.5 + 0.1 * (freqs - 100e9) / 5e9
    return _base("config3_indoor_mimo_100GHz", tri, sid, mats, tx_c, rx_c[None, :], freqs, N, K,
                 gamma=gamma, tx_elem=tx_elem, rx_elem=rx_elem,
                 snr_db=np.arange(0.0, 31.0, 5.0))


# ----------------------------------------------------------------------------
# tiny scenes with closed-form or brute-force answers
# ----------------------------------------------------------------------------

def two_ray(h_tx: float = 10.0, h_rx: float = 2.0, dist: float = 50.0, f: float = 28e9,
            eps_r: float = 5.31, sigma: float = 0.48, rough: float = 0.0, pol: str = "H",
            N: int = 200):
    """Ground plane only (z=0, two triangles over [-1000,1000]^2); Tx at
    (0,0,h_tx), Rx at (dist,0,h_rx): both in the y=0 plane."""
    g = np.array([[[-1000, -1000, 0], [1000, -1000, 0], [1000, 1000, 0]],
                  [[-1000, -1000, 0], [1000, 1000, 0], [-1000, 1000, 0]]], dtype=np.float64)
    tri, sid = _assemble([g])
    return _base("two_ray", tri, sid, [[eps_r, sigma, rough]], (0.0, 0.0, h_tx),
                 [(dist, 0.0, h_rx)], [f], N, 1, pol=pol)


def edge_ceiling(N: int = 20):
    """A ceiling z=10 of two triangles that share the edge x=0 (y in
    [-100,100]; third vertices (+-97.3, 3.1), off any symmetry of the launch
    grid); Tx at the origin, one Rx below it at (30,20,-5), K=1. Every
    launch direction with d_x == 0 exactly (the 4 icosahedron vertices with
    x=0 and the subdivision points of the edge between two of them) that goes
    up meets the ceiling on the shared edge: an edge-ambiguous closest hit by
    construction."""
    ceil = np.array([[[0, -100, 10], [0, 100, 10], [-97.3, 3.1, 10]],
                     [[0, -100, 10], [97.3, 3.1, 10], [0, 100, 10]]], dtype=np.float64)
    tri, sid = _assemble([ceil])
    return _base("edge_ceiling", tri, sid, [[5.31, 0.48, 0.0]], (0.0, 0.0, 0.0),
                 [(30.0, 20.0, -5.0)], [28e9], N, 1)


def corner_reflector(N: int = 150, K: int = 2):
    """Two perpendicular planes: ground z=0 over [-50,20]x[-50,50] and a wall
    x=20 over y in [-50,50], z in [0,60]. Tx (0,0,5), Rx (10,8,3): both in
    front of the wall and above the ground. Up to two reflections there are
    exactly four specular paths: LoS, one off each plane, and one double bounce."""
    ground = np.array([[[-50, -50, 0], [20, -50, 0], [20, 50, 0]],
                       [[-50, -50, 0], [20, 50, 0], [-50, 50, 0]]], dtype=np.float64)
    wall = np.array([[[20, -50, 0], [20, 50, 0], [20, 50, 60]],
                     [[20, -50, 0], [20, 50, 60], [20, -50, 60]]], dtype=np.float64)
    tri, sid = _assemble([ground, wall])
    return _base("corner_reflector", tri, sid, [[5.31, 0.48, 0.0], [3.0, 0.01, 0.0]],
                 (0.0, 0.0, 5.0), [(10.0, 8.0, 3.0)], [28e9], N, K)


def shoebox(N: int = 120, K: int = 3, sub: int = 2, f: float = 60e9, seed: int = 7,
            n_rx: int = 3):
    """Closed room [0,6]x[0,4]x[0,3] with 6 walls split sub x sub; Tx at
    (1.2,1.1,2.1); n_rx receivers drawn U([0.5,5.5]x[0.5,3.5]x[0.5,2.5])
    (seed 7). Per-wall materials cycle through the three config-2 types with
    roughness 0.1 mm."""
    rng = np.random.default_rng(seed)
    groups = [g for _, g in _box_faces((0, 0, 0), (6, 4, 3), sub)]
    types = np.array([[5.31, 0.5, 1e-4], [6.27, 0.1, 1e-4], [3.0, 0.01, 1e-4]])
    mats = np.array([types[s % 3] for s in range(6)])
    tri, sid = _assemble(groups)
    rx = np.column_stack([rng.uniform(0.5, 5.5, n_rx), rng.uniform(0.5, 3.5, n_rx),
                          rng.uniform(0.5, 2.5, n_rx)])
    return _base("shoebox", tri, sid, mats, (1.2, 1.1, 2.1), rx, [f], N, K)


def scene_summary(sc) -> dict:
    return dict(name=sc["name"], T=int(len(sc["tri"])), S=int(len(sc["materials"])),
                n_rx=int(len(sc["rx"])), F=int(len(sc["freqs"])), N=sc["N"], K=sc["K"],
                R=10 * sc["N"] ** 2 + 2, Nt=int(len(sc["tx_elem"])), Nr=int(len(sc["rx_elem"])))


# ----------------------------------------------------------------------------
# batched uneven workload: many Tx-Rx pairs over several scenes
# ----------------------------------------------------------------------------

# subdivisions whose ray counts R = 10 N^2 + 2 are log-spaced over [1e5, 1e7]
BATCH_N_VALUES = np.unique(np.round(np.geomspace(100, 1000, 64)).astype(int))


def batch_scene(s: int, t_min: float = 1e3, t_max: float = 2e5, span: int = 0):
    """Scene s of the batched workload (seed 1000 + s): an urban grid of the
    config-2 kind with nx in [2, 8] x ny in [2, 5] cells, a coarse ground
    (8 x 8 quads) and facade subdivision chosen so that the triangle count is
    close to a target. The target is drawn log-uniform in [t_min, t_max]; with
    span > 0 the targets of scenes 0 .. span-1 are instead the span
    log-spaced values from t_min to t_max, in a seeded order, so that the set
    reaches both ends of the range."""
    rng = np.random.default_rng(1000 + s)
    target = float(np.exp(rng.uniform(np.log(t_min), np.log(t_max))))
    if span > 0:
        order = np.random.default_rng(999).permutation(span)
        target = float(np.geomspace(t_min, t_max, span)[order[s % span]])
    nx = int(rng.integers(2, 9))
    ny = int(rng.integers(2, 6))
    sub = max(1, int(round(np.sqrt(max(target - 128.0, 10.0 * nx * ny) / (10.0 * nx * ny)))))
    sc = config2(N=10, K=1, nx=nx, ny=ny, sub=sub, ground_sub=8, rx_grid=1, seed=1000 + s)
    return dict(tri=sc["tri"], surface_id=sc["surface_id"], materials=sc["materials"], nx=nx, ny=ny,
                seed=1000 + s)


def batch_jobs(scene_list, n_jobs: int = 4096, seed: int = 4, n_values=None, k_range=(2, 8),
               f_exp_range=(6, 10), max_elem_exp: int = 6, tx_exp_range=(0, 3), square_tx: bool = False):
    """Jobs of the batched workload (seed `seed`), each a Tx-Rx pair:
    scene uniform over scene_list; N uniform over n_values (default
    BATCH_N_VALUES, so R is log-uniform over [1e5, 1e7]); K uniform in k_range;
    F = 2^e with e uniform in f_exp_range (64 ... 1024 subcarriers) around a
    carrier from {28, 60, 100, 140, 300} GHz over min(10 GHz, fc / 10); Tx a UPA
    in the y-z plane of 2^a x 2^b elements (a, b uniform in tx_exp_range; b = a
    with square_tx, so (0, 6) gives 1 x 1 ... 64 x 64 UPAs) at a street crossing
    (60 i, 60 j) +- 5 m, height U(5, 30) m; Rx a ULA along y of 2^c elements
    (c in [0, max_elem_exp]) in an x-street (60 i +- 8 m), height 1.5 m, so that
    neither end is inside a building; element spacing half a carrier
    wavelength; polarisation V or H; gamma = 5 dB/km x (f / 300 GHz)
    (synthetic stand-in for Eq. 9)."""
    rng = np.random.default_rng(seed)
    n_values = BATCH_N_VALUES if n_values is None else np.asarray(n_values)
    carriers = np.array([28e9, 60e9, 100e9, 140e9, 300e9])
    jobs = []
    for _ in range(n_jobs):
        s = int(rng.integers(0, len(scene_list)))
        sc = scene_list[s]
        nx, ny = sc["nx"], sc["ny"]
        N = int(rng.choice(n_values))
        K = int(rng.integers(k_range[0], k_range[1] + 1))
        F = int(2 ** rng.integers(f_exp_range[0], f_exp_range[1] + 1))
        fc = float(rng.choice(carriers))
        bw = min(10e9, fc / 10.0)
        freqs = fc + (np.arange(F) - F // 2) * (bw / F)
        lam = 299792458.0 / fc
        tx = np.array([60.0 * rng.integers(1, nx) + rng.uniform(-5, 5),
                       60.0 * rng.integers(1, ny) + rng.uniform(-5, 5), rng.uniform(5, 30)])
        rx = np.array([60.0 * rng.integers(0, nx + 1) + rng.uniform(-8, 8),
                       rng.uniform(-10.0, 60.0 * ny + 10.0), 1.5])
        nty, ntz = int(2 ** rng.integers(tx_exp_range[0], tx_exp_range[1] + 1)), \
            int(2 ** rng.integers(tx_exp_range[0], tx_exp_range[1] + 1))
        if square_tx:
            ntz = nty
        nr = int(2 ** rng.integers(0, max_elem_exp + 1))
        pol = "V" if rng.integers(0, 2) == 0 else "H"
        jobs.append(dict(scene=s, N=N, K=K, tx=tx, rx=rx, freqs=freqs, pol=pol,
                         gamma=(5.0 * freqs / 300e9).astype(np.float32),
                         tx_elem=upa_yz(tx, nty, ntz, lam / 2), rx_elem=ula_y(rx, nr, lam / 2)))
    return jobs


def batch_job_scene(scene, job) -> dict:
    """One job as a single-receiver scene dict (for the oracle and the per-pair API)."""
    return _base("batch_job", scene["tri"], scene["surface_id"], scene["materials"], job["tx"],
                 [job["rx"]], job["freqs"], job["N"], job["K"], pol=job["pol"], gamma=job["gamma"],
                 tx_elem=job["tx_elem"], rx_elem=job["rx_elem"])
