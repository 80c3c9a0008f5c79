"""CPU-only checks of the C-ABI library: it loads, exports every symbol the
header declares, and its host-only octree builder matches the oracle's
independent rebuild bit for bit.  No GPU compute is called here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import octaoctree_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_08469_gb300 import build
    build.build()
    from paper_2606_08469_gb300 import _lib
    return _lib.load()


def _declared_functions():
    import glob
    names = []
    for path in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        txt = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \t\*]*?\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", txt,
                            flags=re.M)
    return sorted(set(names))


def test_header_symbols_exported(lib):
    names = _declared_functions()
    assert {"octree_build", "octa_query_fwd", "octa_query_bwd", "residual_loss",
            "adam_step", "octa_measure_ffma", "octa_measure_mma"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    from paper_2606_08469_gb300 import _lib
    assert set(_lib._SIGNATURES) >= set(names)


def test_measure_mma_validation_without_gpu(lib):
    """octa_measure_mma checks its arguments on the host before any launch."""
    from paper_2606_08469_gb300 import _lib as L
    buf = (C.c_int64 * 3)()
    ptr = C.cast(buf, C.c_void_p)
    assert lib.octa_measure_mma(None, 64, 4, 5, 1, None) == L.OCTA_EINVAL
    for n, k, reps, iss in ((8, 4, 5, 1), (72, 4, 5, 1), (272, 4, 5, 1), (64, 0, 5, 1),
                            (64, 9, 5, 1), (64, 4, 1, 1), (64, 4, 5, 3), (64, 4, 5, 0)):
        assert lib.octa_measure_mma(ptr, n, k, reps, iss, None) == L.OCTA_EINVAL, (n, k, reps, iss)


def test_struct_sizes_match_header(lib):
    """The ctypes mirrors have the C layout (checked through a sizing call)."""
    from paper_2606_08469_gb300 import _lib as L
    assert C.sizeof(L.octa_tree_desc) == 4 + 4 + 8 + 4 * 16 + 4 * 17 + 4 + 8 * 17
    assert lib.octa_abi_version() == 8
    assert C.sizeof(L.octa_prims) == 8 + 8 + 4 + 4
    assert C.sizeof(L.octa_queries) == 8 + 8 + 8 + 8 * 17 + 8 + 8 + 8 + 4 + 4 + 8
    assert C.sizeof(L.octa_predictor) == 8 + 8 + 8 + 4 + 4 + 4 * 16
    assert C.sizeof(L.octa_pairs) == 6 * 8 + 8 + 8 * 17 + 8 * 16 + 6 * 8


@pytest.mark.parametrize("seed,depth,R", [
    (1000, 4, [16, 16, 8, 8, 8]),
    (1001, 6, [32, 32, 16, 16, 8, 8, 8]),
    (1002, 8, [64, 64, 32, 32, 16, 16, 8, 8, 8]),
    (1403, 7, [64, 64, 32, 32, 16, 16, 8, 8]),
    (1407, 9, [64, 64, 32, 32, 16, 16, 8, 8, 8, 8]),
    (0, 0, [4]),
])
def test_octree_build_matches_oracle(lib, seed, depth, R):
    from paper_2606_08469_gb300 import api
    t = api.octree_build(seed, depth, 0.6, R)
    o = O.build_tree(seed, depth, 0.6, R)
    assert t.num_nodes == o.num_nodes and t.num_texels == o.num_texels
    np.testing.assert_array_equal(t.first_child, o.first_child)
    np.testing.assert_array_equal(t.node_coord, o.node_coord)
    np.testing.assert_array_equal(t.map_offset, o.map_offset)
    np.testing.assert_array_equal(t.level_node_start, o.level_node_start)
    np.testing.assert_array_equal(t.level_texel_base, o.level_texel_base)


def test_octree_dense_and_flags(lib):
    from paper_2606_08469_gb300 import api
    t = api.octree_build(5, 3, 1.0, [2, 2, 2, 2])     # p = 1: full octree
    assert t.num_nodes == 1 + 8 + 64 + 512
    flags = [1, 0, 0, 1, 0, 0, 0, 0, 0]
    t = api.octree_from_flags(flags, 2, [4, 2, 2])
    o = O.tree_from_flags(flags, 2, [4, 2, 2])
    np.testing.assert_array_equal(t.first_child, o.first_child)
    np.testing.assert_array_equal(t.map_offset, o.map_offset)
    t = api.octree_from_flags([], 3, [2, 2, 2, 2])     # root only
    assert t.num_nodes == 1 and t.num_texels == 4


def test_octree_errors(lib):
    from paper_2606_08469_gb300 import _lib as L
    desc = L.octa_tree_desc()
    R = (C.c_int32 * 3)(4, 1, 4)
    assert lib.octree_build(1, 2, 0.6, R, C.byref(desc), None, None, None) == L.OCTA_ERANGE
    assert b"R[1]" in lib.octa_last_error()
    R = (C.c_int32 * 3)(4, 4, 4)
    assert lib.octree_build(1, 2, 1.5, R, C.byref(desc), None, None, None) == L.OCTA_EINVAL
    assert lib.octree_build(1, 16, 0.5, R, C.byref(desc), None, None, None) == L.OCTA_ERANGE
    assert lib.octree_build(1, 2, 0.5, None, C.byref(desc), None, None, None) == L.OCTA_EINVAL
    assert lib.octree_build(1, 2, 0.5, R, C.byref(desc), None, None, None) == L.OCTA_OK
    assert lib.octree_from_flags(None, 3, 2, R, C.byref(desc), None, None, None) == L.OCTA_EINVAL


def test_query_validation_without_gpu(lib):
    """Argument checks run on the host before any launch."""
    from paper_2606_08469_gb300 import _lib as L
    q = L.octa_queries()
    q.n = 0
    s = L.octa_scene()
    # NULL scenes / queries
    assert lib.octa_query_fwd(None, 1, C.byref(q), None, None, None, None, None) == L.OCTA_EINVAL
    # zero scenes
    assert lib.octa_query_fwd(C.byref(s), 0, C.byref(q), None, None, None, None, None) == L.OCTA_ERANGE
    # scene with NULL arrays
    q.scene_start[1] = 0
    assert lib.octa_query_fwd(C.byref(s), 1, C.byref(q), None, None, None, None, None) == L.OCTA_EINVAL
    assert b"NULL" in lib.octa_last_error()
    # residual_loss: bad sizes and NULLs
    assert lib.residual_loss(None, None, None, None, 0, C.c_float(0.01), 1, None, None, None, None,
                             None, 0, None) == L.OCTA_EINVAL
    assert lib.octa_workspace_bytes(L.OCTA_OP_LOSS, 100) >= 8 * 1024
    assert lib.octa_workspace_bytes(99, 100) == 0


def test_tuning_knobs_round_trip(lib):
    from paper_2606_08469_gb300 import autotune as T
    T.set_tuning({"fwd_ctas_per_sm": 3, "train_order": 1})
    got = T.get_tuning()
    assert got["fwd_ctas_per_sm"] == 3 and got["train_order"] == 1 and got["fwd_order"] == 0
    from paper_2606_08469_gb300 import _lib as L
    bad = L.octa_tuning()
    bad.fwd_order = 7
    assert lib.octa_set_tuning(C.byref(bad)) == L.OCTA_EINVAL
    for field, value in (("gather_stages", 5), ("l1_carveout", 3), ("fwd_run", 65)):
        bad = L.octa_tuning()
        setattr(bad, field, value)
        assert lib.octa_set_tuning(C.byref(bad)) == L.OCTA_EINVAL, field
    T.set_tuning({"gather_stages": 3, "l1_carveout": 1})
    got = T.get_tuning()
    assert got["gather_stages"] == 3 and got["l1_carveout"] == 1
    assert C.sizeof(L.octa_tuning) == 12 * 4
    T.set_tuning(None)
    assert all(v == 0 for v in T.get_tuning().values())


def test_training_regime_and_predictor_validation_without_gpu(lib):
    """The tracer's, the M-sample loss's and the predictor's argument checks
    run on the host before any launch (no device needed)."""
    from paper_2606_08469_gb300 import _lib as L
    # tracer: NULL scene, too many primitives, rays_per_origin < 1, t_min < 0
    assert lib.octa_trace_rays(None, None, 1, None, 0, C.c_float(1e-4), None, None, None, None,
                               None) == L.OCTA_EINVAL
    pr = L.octa_prims()
    pr.n_planes = L.OCTA_MAX_PRIMS + 1
    assert lib.octa_trace_rays(C.byref(pr), None, 1, None, 0, C.c_float(1e-4), None, None, None,
                               None, None) == L.OCTA_ERANGE
    pr.n_planes = 0
    assert lib.octa_trace_rays(C.byref(pr), None, 0, None, 0, C.c_float(1e-4), None, None, None,
                               None, None) == L.OCTA_EINVAL
    assert lib.octa_trace_rays(C.byref(pr), None, 1, None, 0, C.c_float(-1.0), None, None, None,
                               None, None) == L.OCTA_EINVAL
    assert lib.octa_trace_rays(C.byref(pr), None, 1, None, 0, C.c_float(1e-4), None, None, None,
                               None, None) == L.OCTA_OK                     # empty batch
    pr.n_spheres = 2                                                       # NULL sphere array
    assert lib.octa_trace_rays(C.byref(pr), None, 1, None, 0, C.c_float(1e-4), None, None, None,
                               None, None) == L.OCTA_EINVAL
    # M-sample loss: no pairs, no samples, NULL arrays
    assert lib.residual_loss_multi(None, None, None, None, 0, 4, C.c_float(0.01), 0, None, None,
                                   None, None, None, 0, None) == L.OCTA_EINVAL
    assert lib.residual_loss_multi(None, None, None, None, 10, 0, C.c_float(0.01), 0, None, None,
                                   None, None, None, 0, None) == L.OCTA_EINVAL
    assert lib.residual_loss_multi(None, None, None, None, 10, 4, C.c_float(0.01), 0, None, None,
                                   None, None, None, 0, None) == L.OCTA_EINVAL
    # predictor: levels, table size, NULL arrays, the tensor-core level limit
    p = L.octa_predictor()
    q = L.octa_queries()
    q.n = 0
    p.levels = 0
    assert lib.octa_disparity(C.byref(p), C.byref(q), None, None) == L.OCTA_ERANGE
    p.levels, p.log2_T = 2, 30
    assert lib.octa_disparity(C.byref(p), C.byref(q), None, None) == L.OCTA_ERANGE
    p.log2_T = 12
    assert lib.octa_disparity(C.byref(p), C.byref(q), None, None) == L.OCTA_EINVAL
    p.table = p.weights = 64                     # never dereferenced: n = 0
    assert lib.octa_disparity(C.byref(p), C.byref(q), None, None) == L.OCTA_OK
    p.levels, p.weights_bf16 = 15, 64
    q.n = 5
    assert lib.octa_disparity(C.byref(p), C.byref(q), None, None) == L.OCTA_ERANGE


def test_query_attribute_and_form_validation_without_gpu(lib):
    """Eq. 12's attribute count and the query forms are validated on the host."""
    from paper_2606_08469_gb300 import _lib as L
    q = L.octa_queries()
    q.n = 0
    q.n_attrs = L.OCTA_MAX_ATTRS + 1
    s = L.octa_scene()
    assert lib.octa_query_fwd(C.byref(s), 1, C.byref(q), None, None, None, None, None) == L.OCTA_ERANGE
    assert b"n_attrs" in lib.octa_last_error()
