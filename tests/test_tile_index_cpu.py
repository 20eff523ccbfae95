"""The index arithmetic of the 3D stage kernels' tiles, checked on the CPU.

The 3D stage kernels walk three cell sets of a TX x TY x TZ tile through
host-and-device functions of ``csrc/dg_common.cuh``: ``ring3d_cell`` (the cells
whose slopes the min/max limiter of Sec. 2.5 must limit: the tile and its six
face slabs, whose records the face Gauss points read), ``halo3d_cell`` (the cells
whose centroid primitives that limiter reads: the halo-1 box and one more layer
beyond each face), and ``div_by_magic`` (the face loop's division by a run-time
face count).  This test compiles them for the host with nvcc, for every tile
shape the kernels instantiate, and checks that every index stays inside its
shared-memory box, that no cell is listed twice, that the primitives cover every
neighbour the limiter reads and the ring covers every cell a face reads, and that
the multiply-high division is exact over the whole range the kernels use.  No GPU
is needed.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1305_5536_gb300", "csrc")

# tile shapes of the 3D stage kernels (Euler: FP32 8x8x4, 8x4x4; FP64 4x4x4,
# 8x4x2; MHD: FP32 8x4x4, 8x8x4; FP64 4x4x4)
SHAPES = [(8, 8, 4), (8, 4, 4), (4, 4, 4), (8, 4, 2)]

_SRC = r"""
#include "dg_common.cuh"
template <int TX, int TY, int TZ>
static int cells(int which, int* out) {
  const int n = which == 0 ? dgk::ring3d_count<TX, TY, TZ>() : dgk::halo3d_count<TX, TY, TZ>();
  for (int e = 0; e < n; ++e) {
    int x, y, z;
    if (which == 0) dgk::ring3d_cell<TX, TY, TZ>(e, x, y, z);
    else dgk::halo3d_cell<TX, TY, TZ>(e, x, y, z);
    out[3 * e] = x; out[3 * e + 1] = y; out[3 * e + 2] = z;
  }
  return n;
}
extern "C" int tile_cells(int shape, int which, int* out) {
  switch (shape) {
    case 0: return cells<8, 8, 4>(which, out);
    case 1: return cells<8, 4, 4>(which, out);
    case 2: return cells<4, 4, 4>(which, out);
    case 3: return cells<8, 4, 2>(which, out);
  }
  return -1;
}
// mismatches of floor(n / d) by multiply-high over 0 <= n < nmax, 2 <= d <= dmax
extern "C" long magic_mismatches(int nmax, int dmax) {
  long bad = 0;
  for (int d = 2; d <= dmax; ++d) {
    const unsigned m = dgk::div_magic((unsigned)d);
    for (int n = 0; n < nmax; ++n) bad += dgk::div_by_magic(n, m) != n / d;
  }
  return bad;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and not shutil.which(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("tileidx")
    src = d / "tileidx.cu"
    src.write_text(_SRC)
    so = d / "libtileidx.so"
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                    "-shared", "-I", CSRC, str(src), "-o", str(so)], check=True,
                   capture_output=True)
    L = ctypes.CDLL(str(so))
    L.tile_cells.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    L.tile_cells.restype = ctypes.c_int
    L.magic_mismatches.argtypes = [ctypes.c_int, ctypes.c_int]
    L.magic_mismatches.restype = ctypes.c_long
    return L


def _cells(L, shape, which):
    out = np.zeros((4096, 3), dtype=np.int32)
    n = L.tile_cells(shape, which, out.ctypes.data)
    return [tuple(int(v) for v in c) for c in out[:n]]


AXES = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


@pytest.mark.parametrize("k", range(len(SHAPES)), ids=["%dx%dx%d" % s for s in SHAPES])
def test_ring_is_the_tile_and_its_face_slabs(lib, k):
    TX, TY, TZ = SHAPES[k]
    ring = _cells(lib, k, 0)
    assert len(set(ring)) == len(ring)
    # halo-1 box coordinates: the tile is 1..T, the box 0..T+1
    for x, y, z in ring:
        assert 0 <= x <= TX + 1 and 0 <= y <= TY + 1 and 0 <= z <= TZ + 1
        outside = (x in (0, TX + 1)) + (y in (0, TY + 1)) + (z in (0, TZ + 1))
        assert outside <= 1, (x, y, z)  # no edge or corner of the box
    tile = {(x, y, z) for x in range(1, TX + 1) for y in range(1, TY + 1)
            for z in range(1, TZ + 1)}
    # every face of the tile joins a tile cell to its neighbour along the axis:
    # both are limited
    read = {(x + a, y + b, z + c) for (x, y, z) in tile for (a, b, c) in AXES} | tile
    assert read == set(ring)


@pytest.mark.parametrize("k", range(len(SHAPES)), ids=["%dx%dx%d" % s for s in SHAPES])
def test_halo_primitives_cover_every_limiter_neighbour(lib, k):
    TX, TY, TZ = SHAPES[k]
    R1X, R1Y, R1Z = TX + 2, TY + 2, TZ + 2
    halo = _cells(lib, k, 1)
    assert len(set(halo)) == len(halo)
    for x, y, z in halo:  # halo-2 box coordinates
        assert 0 <= x < TX + 4 and 0 <= y < TY + 4 and 0 <= z < TZ + 4
    # the first R1 cells are the halo-1 box in its own row-major order (the
    # kernels store the averages of cell e at halo-1 index e)
    for e in range(R1X * R1Y * R1Z):
        x, y, z = halo[e]
        assert ((z - 1) * R1Y + (y - 1)) * R1X + (x - 1) == e
    # the limiter reads, for every ring cell, its own and its six neighbours'
    # primitives (ring in halo-1 coordinates = halo-2 coordinates - 1)
    need = set()
    for (x, y, z) in _cells(lib, k, 0):
        X, Y, Z = x + 1, y + 1, z + 1
        need.add((X, Y, Z))
        need |= {(X + a, Y + b, Z + c) for (a, b, c) in AXES}
    assert need <= set(halo)
    # and nothing else but the 8 corners of the halo-1 box
    extra = set(halo) - need
    assert len(extra) == 8 and all(x in (1, TX + 2) and y in (1, TY + 2) and z in (1, TZ + 2)
                                   for x, y, z in extra)


def test_multiply_high_division_is_exact_over_the_kernels_range(lib):
    # face indices below 2^14; the divisors are the face counts of a row (TX or
    # TX + 1) and of a plane, between 2 and 1024 for every tile shape
    for TX, TY, TZ in SHAPES:
        for d in range(3):
            FX, FY, FZ = TX + (d == 0), TY + (d == 1), TZ + (d == 2)
            assert 2 <= FX and FX * FY <= 1024 and FX * FY * FZ < 1 << 14
    assert lib.magic_mismatches(1 << 14, 1024) == 0
