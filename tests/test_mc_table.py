"""The library's marching-cubes case table (generated on the host, krig_marching_cubes_table)
against the oracle's case triangulation, derived independently from the cube's geometry, for all
256 corner configurations; and the host-side argument checks of krig_marching_cubes.  CPU only."""
import ctypes

import numpy as np

from oracle import downstream as ds
from paper_2303_09523_gb300 import binding


def test_case_table_matches_oracle_for_every_configuration():
    tri, nt = binding.marching_cubes_table()
    for c in range(256):
        # corner i = dx + 2 dy + 4 dz of the library is the oracle's offset (dx, dy, dz)
        inside = {(i & 1, (i >> 1) & 1, i >> 2): bool((c >> i) & 1) for i in range(8)}
        exp = ds.mc_case_triangles(inside)
        got = [tuple(int(e) for e in tri[c, 3 * q:3 * q + 3]) for q in range(int(nt[c]))]
        assert got == exp, c
        assert all(int(e) == -1 for e in tri[c, 3 * int(nt[c]):])


def test_marching_cubes_rejects_before_any_launch():
    L = binding.lib()
    vp = ctypes.c_void_p
    n = vp(256)
    assert L.krig_marching_cubes(None, 4, 4, 4, 0.5, vp(256), 10, n, vp(256), 1 << 20, None) == binding.KRIG_EINVAL
    assert L.krig_marching_cubes(vp(256), 1, 4, 4, 0.5, vp(256), 10, n, vp(256), 1 << 20, None) == binding.KRIG_EINVAL
    assert L.krig_marching_cubes(vp(256), 4, 4, 4, 0.5, None, 10, n, vp(256), 1 << 20, None) == binding.KRIG_EINVAL
    assert L.krig_marching_cubes(vp(256), 4, 4, 4, float("nan"), vp(256), 10, n, vp(256), 1 << 20,
                                 None) == binding.KRIG_EINVAL
    need = L.krig_marching_cubes_workspace_bytes(5, 6, 7)
    assert need >= 4 * 5 * 6
    assert L.krig_marching_cubes(vp(256), 5, 6, 7, 0.5, vp(256), 10, n, vp(256), need - 1,
                                 None) == binding.KRIG_EWORKSPACE
    assert L.krig_marching_cubes_workspace_bytes(1, 6, 7) == 0
