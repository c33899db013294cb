"""Jittered-lattice periodic Voronoi meshes (host input of the radiation step).

Mesh-generating points are lattice sites plus a seeded uniform jitter
(Sec. 3.3 and 3.6 perturb a regular lattice the same way).  The tessellation
is computed by the native builder in voronoi.cpp.
"""
import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voronoi.cpp")
_LIB = os.path.join(_HERE, "libvoronoi.so")
_lock = threading.Lock()
_lib = None


def build_voronoi_lib(force: bool = False) -> str:
    """Compile voronoi.cpp into libvoronoi.so next to it (host C++, no CUDA)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-pthread",
                                   _SRC, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _get_lib():
    global _lib
    if _lib is None:
        build_voronoi_lib()
        lib = ctypes.CDLL(_LIB)
        lib.vor_build_lattice.restype = ctypes.c_void_p
        lib.vor_build_lattice.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.vor_sizes.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int64)] * 3
        lib.vor_fetch.argtypes = [ctypes.c_void_p] * 10
        lib.vor_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class Mesh:
    """Periodic Voronoi mesh in plain numpy arrays (float64 / int32 / int64).

    face_normal points from generator i to generator j; face_w is the face
    velocity (zero for a static mesh).  cell_face_idx holds f when the cell
    is the face's first cell and -(f+1) when it is the second.
    """
    n: tuple
    box: np.ndarray
    points: np.ndarray
    cell_volume: np.ndarray
    cell_centroid: np.ndarray
    face_cells: np.ndarray
    face_shift: np.ndarray
    face_area: np.ndarray
    face_normal: np.ndarray
    face_centroid: np.ndarray
    cell_face_ptr: np.ndarray
    cell_face_idx: np.ndarray
    face_w: np.ndarray = field(default=None)

    @property
    def n_cells(self) -> int:
        return int(self.cell_volume.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.face_area.shape[0])

    def face_offset(self):
        """[Nf, 2, 3]: the face centroid relative to each of the face's two
        cells, x_f - x_i and x_f - x_j', where j' is the periodic image of j
        that meets i across the face (face centroids are in cell i's frame,
        j' = x_j + shift * box)."""
        i, j = self.face_cells[:, 0], self.face_cells[:, 1]
        xj = self.cell_centroid[j] + self.face_shift.astype(np.float64) * self.box
        off = np.empty((self.n_faces, 2, 3))
        off[:, 0] = self.face_centroid - self.cell_centroid[i]
        off[:, 1] = self.face_centroid - xj
        return off

    def face_velocity(self, w_gen):
        """[Nf, 3] face velocities from the velocities w_gen [N, 3] of the
        mesh-generating points (the face-velocity equation of Sec. 2.2): the
        mean velocity of the face's two generators, plus the velocity along
        r_j - r_i that the relative motion of the generators gives the point
        of the face at its centroid x_f,
          w_f = [(w_i - w_j) . (x_f - (r_i + r_j) / 2) / |r_j - r_i|] (r_j - r_i) / |r_j - r_i|
                + (w_i + w_j) / 2,
        with r_j the periodic image of generator j that faces i (x_f is in
        cell i's frame)."""
        w_gen = np.asarray(w_gen, np.float64)
        i, j = self.face_cells[:, 0], self.face_cells[:, 1]
        ri = self.points[i]
        rj = self.points[j] + self.face_shift.astype(np.float64) * self.box
        d = rj - ri
        L = np.linalg.norm(d, axis=1)
        e = d / L[:, None]
        s = np.sum((w_gen[i] - w_gen[j]) * (self.face_centroid - 0.5 * (ri + rj)), axis=1) / L
        return np.ascontiguousarray(s[:, None] * e + 0.5 * (w_gen[i] + w_gen[j]))

    def lattice_index(self):
        """(ix, iy, iz) lattice coordinates of every cell."""
        nx, ny, nz = self.n
        c = np.arange(self.n_cells)
        return c // (ny * nz), (c // nz) % ny, c % nz


def jittered_lattice(n, box=(1.0, 1.0, 1.0), jitter=0.25, seed=0):
    """Lattice sites ((i + 0.5) h) displaced by U(-jitter, jitter) * h per axis."""
    nx, ny, nz = n
    box = np.asarray(box, dtype=np.float64)
    h = box / np.array([nx, ny, nz], dtype=np.float64)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    base = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-jitter, jitter, size=base.shape)
    pts = (base + 0.5 + jit) * h
    return np.ascontiguousarray(pts), jitter * h


def build_mesh(n, box=(1.0, 1.0, 1.0), jitter=0.25, seed=0, threads=0) -> Mesh:
    """Periodic Voronoi mesh of an n[0] x n[1] x n[2] jittered lattice."""
    n = tuple(int(v) for v in n)
    pts, jit = jittered_lattice(n, box, jitter, seed)
    # guard the bound used by the builder's search: jitter strictly inside it
    jit = np.ascontiguousarray(np.asarray(jit, dtype=np.float64) * (1 + 1e-9) + 1e-300)
    box = np.ascontiguousarray(np.asarray(box, dtype=np.float64))
    lib = _get_lib()
    h = lib.vor_build_lattice(pts.ctypes.data, n[0], n[1], n[2], box.ctypes.data, jit.ctypes.data,
                              int(threads))
    if not h:
        raise RuntimeError("voronoi builder rejected its arguments")
    try:
        nc, nf, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib.vor_sizes(h, ctypes.byref(nc), ctypes.byref(nf), ctypes.byref(nnz))
        nc, nf, nnz = nc.value, nf.value, nnz.value
        vol = np.empty(nc); cen = np.empty((nc, 3))
        fcells = np.empty((nf, 2), np.int32); fshift = np.empty((nf, 3), np.int8)
        farea = np.empty(nf); fnorm = np.empty((nf, 3)); fcen = np.empty((nf, 3))
        ptr = np.empty(nc + 1, np.int64); idx = np.empty(nnz, np.int32)
        lib.vor_fetch(h, vol.ctypes.data, cen.ctypes.data, fcells.ctypes.data, fshift.ctypes.data,
                      farea.ctypes.data, fnorm.ctypes.data, fcen.ctypes.data, ptr.ctypes.data,
                      idx.ctypes.data)
    finally:
        lib.vor_free(h)
    return Mesh(n=n, box=box, points=pts, cell_volume=vol, cell_centroid=cen, face_cells=fcells,
                face_shift=fshift, face_area=farea, face_normal=fnorm, face_centroid=fcen,
                cell_face_ptr=ptr, cell_face_idx=idx, face_w=np.zeros((nf, 3)))
