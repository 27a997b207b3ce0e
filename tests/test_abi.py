"""CPU checks of the C ABI boundary: the library loads without a GPU and exports
every function that include/pfasst_mg.h declares; host-side validation works."""
import ctypes
import os
import re

import pytest

import paper_1407_6486_gb300 as pmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(pfasst_mg_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1407_6486_gb300 import _build
    _build.build()
    return pmg.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(pmg.EXPORTS) | declared


def test_default_options(lib):
    o = pmg.pfasst_mg_default_options()
    assert o.nu1 == 2 and o.nu2 == 1 and o.vcycles == 2 and abs(o.omega - 2 / 3) < 1e-15
    assert o.interp_order == 4 and o.precision == pmg.PMG_PREC_FP64
    assert o.slice_groups == 0 and o.vcycle_tail == -1 and o.coarse_vcycles == -1 and o.single_grid_vcycle == 0


def _ws(dim, n, sf, nl, sc, P, **kw):
    o = pmg.pfasst_mg_default_options(**kw)
    return pmg.pfasst_mg_workspace_bytes(pmg.pmg_grid(dim, n), pmg.pmg_nodes_desc(sf, 0),
                                         pmg.pmg_levels(nl, pmg.pmg_nodes_desc(sc, 0)), P, o)


def test_workspace_size_grows_with_problem(lib):
    a = _ws(2, 31, 5, 2, 3, 4)
    b = _ws(2, 63, 5, 2, 3, 4)
    c = _ws(2, 63, 5, 2, 3, 8)
    assert 0 < a < b < c
    # FP64 fine state alone: U and q over slices and nodes, padded rows
    assert b >= 8 * 64 * 63 * (5 + 4) * 4
    # mixed precision halves the multigrid scratch
    assert _ws(3, 31, 5, 2, 3, 4, precision=1) < _ws(3, 31, 5, 2, 3, 4, precision=0)


def test_fixed_vcycle_counts_plan_no_fine_F(lib):
    """With a fixed V-cycle count the fine level stores no F = A U (the end-of-iteration
    pass and the FAS restriction evaluate it from U): the workspace is smaller than the
    full-solve one by exactly one FP64 array of slices x nodes padded grids."""
    for dim, n, sf, P in ((2, 63, 5, 4), (3, 31, 5, 8), (3, 63, 3, 2)):
        full = _ws(dim, n, sf, 2, 3, P, vcycles=0)
        fixed = _ws(dim, n, sf, 2, 3, P, vcycles=2)
        fbytes = 8 * (n + 1) * n ** (dim - 1) * P * sf
        assert full - fixed == (fbytes + 255) // 256 * 256, (dim, n, full, fixed)


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(n=30), dict(n=1), dict(sf=1), dict(sf=12), dict(nl=3),
    dict(sc=7), dict(P=0), dict(n=3, nl=2),
])
def test_invalid_descriptions_are_rejected(lib, bad):
    p = dict(dim=2, n=31, sf=5, nl=2, sc=3, P=4)
    p.update(bad)
    with pytest.raises(pmg.PMGError) as ei:
        _ws(p["dim"], p["n"], p["sf"], p["nl"], p["sc"], p["P"])
    assert ei.value.code in (pmg.PMG_ERR_INVALID_ARG, pmg.PMG_ERR_UNSUPPORTED)
    assert pmg.pfasst_mg_last_error()


@pytest.mark.parametrize("opt", [dict(smoother=5), dict(nu1=0, nu2=0), dict(precision=3),
                                 dict(interp_order=3), dict(omega=0.0), dict(vcycles=-1),
                                 dict(coarse_vcycles=-2), dict(coarse_vcycles=0, mg_tol=0.0),
                                 dict(vcycle_tail=2), dict(vcycle_tail=-2)])
def test_invalid_options_are_rejected(lib, opt):
    with pytest.raises(pmg.PMGError) as ei:
        _ws(2, 31, 5, 2, 3, 4, **opt)
    assert ei.value.code == pmg.PMG_ERR_INVALID_ARG


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.pfasst_mg_predict(None) == pmg.PMG_ERR_INVALID_ARG
    assert lib.pfasst_mg_sweep(None, 0) == pmg.PMG_ERR_INVALID_ARG
    assert lib.pfasst_mg_destroy(None) == pmg.PMG_OK
    assert lib.pfasst_mg_launch_count(None) == -1


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1407_6486_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "pfasst_oracle" not in src and "orc_" not in src, f


def test_create_rejects_nested_nodes_that_do_not_nest(lib):
    """5 Gauss-Lobatto nodes are not a subset of 9 (only odd counts share the midpoint
    with 3); the coarse level needs coincident nodes for point-wise restriction in time."""
    h = ctypes.c_void_p()
    o = pmg.pfasst_mg_default_options()
    rc = lib.pfasst_mg_create(ctypes.byref(pmg.pmg_grid(1, 63)), ctypes.byref(pmg.pmg_nodes_desc(9, 0)),
                              ctypes.byref(pmg.pmg_levels(2, pmg.pmg_nodes_desc(5, 0))), 1.0, 0.01, 2,
                              ctypes.byref(o), None, None, 0, ctypes.byref(h))
    assert rc == pmg.PMG_ERR_INVALID_ARG and not h.value
    assert "subset" in pmg.pfasst_mg_last_error()


def test_batch_validation_reports_the_bad_problem(lib):
    good = pmg.pmg_problem_desc(pmg.pmg_grid(2, 31), 3, 1.0, 0.01)
    bad = pmg.pmg_problem_desc(pmg.pmg_grid(2, 30), 3, 1.0, 0.01)
    o = pmg.pfasst_mg_default_options()
    assert pmg.pfasst_mg_batch_workspace_bytes([good, good], o) > 0
    with pytest.raises(pmg.PMGError) as ei:
        pmg.pfasst_mg_batch_workspace_bytes([good, bad], o)
    assert "problem 1" in str(ei.value)
    with pytest.raises(pmg.PMGError) as ei:
        pmg.pfasst_mg_batch_workspace_bytes([good], pmg.pfasst_mg_default_options(vcycles=0))
    assert ei.value.code == pmg.PMG_ERR_UNSUPPORTED


def test_uneven_workload_recipe():
    from paper_1407_6486_gb300 import inputs
    probs = inputs.heat_uneven_c4()
    assert len(probs) == 64 and sum(p.dim == 2 for p in probs) == 32
    assert {p.n for p in probs if p.dim == 2} <= {63, 127, 255, 511}
    assert {p.n for p in probs if p.dim == 3} <= {31, 63, 127}
    assert all(0.1 <= p.nu <= 2 and 1e-3 <= p.dt <= 1e-2 and p.nodes in (3, 5) for p in probs)


def test_network_parameter_layout_and_host_init(lib):
    import numpy as np
    assert pmg.pfasst_mg_net_param_count() == pmg.NET_PARAMS == 16 * 27 + 16 + 16 * 27 * 16 + 16 + 27 * 16 + 1
    p = pmg.pfasst_mg_net_init(5)
    q = pmg.pfasst_mg_net_init(5)
    assert np.array_equal(p, q) and not np.array_equal(p, pmg.pfasst_mg_net_init(6))
    w1, b1 = p[:432], p[432:448]
    w2, b2 = p[448:7360], p[7360:7376]
    w3, b3 = p[7376:7808], p[7808:]
    assert not b1.any() and not b2.any() and not b3.any()
    # He scaling: std sqrt(2/27), sqrt(2/432), sqrt(1/432) within sampling error
    for w, sd in ((w1, (2 / 27) ** 0.5), (w2, (2 / 432) ** 0.5), (w3, (1 / 432) ** 0.5)):
        assert abs(w.std() / sd - 1) < 4 / len(w) ** 0.5 + 0.02 and abs(w.mean()) < 4 * sd / len(w) ** 0.5


def test_network_argument_validation_needs_no_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.pfasst_mg_net_create(0, 16, None, ctypes.byref(h)) == pmg.PMG_ERR_INVALID_ARG
    assert lib.pfasst_mg_net_create(1, 2, None, ctypes.byref(h)) == pmg.PMG_ERR_INVALID_ARG
    assert lib.pfasst_mg_net_create(1, 300, None, ctypes.byref(h)) == pmg.PMG_ERR_INVALID_ARG
    assert "n <= 255" in pmg.pfasst_mg_net_last_error(None)
    assert lib.pfasst_mg_net_init(None, 1) == pmg.PMG_ERR_INVALID_ARG
    assert lib.pfasst_mg_net_train(None, 1, 1e-3, 0, 0.1, 0.15, 0, 2, 0, None) == pmg.PMG_ERR_INVALID_ARG
    assert lib.pfasst_mg_set_smoother_net(None, None, 15, 1, None, None, None) == pmg.PMG_ERR_INVALID_ARG
    assert lib.pfasst_mg_net_destroy(None) == pmg.PMG_OK


def test_every_kernel_identifier_has_a_name(lib):
    names = []
    k = 0
    while True:
        raw = lib.pfasst_mg_kernel_name(k)
        assert raw is not None, k
        if raw.decode() == "unknown":
            break
        names.append(raw.decode())
        k += 1
    assert len(names) == len(set(names)) and len(names) >= 30
    assert {"net_layer2_mma", "net_layer2_mma_bwd", "net_wgrad", "fine_rhs_residual"} <= set(names)
    assert lib.pfasst_mg_kernel_name(-1).decode() == "unknown"


def test_slice_groups_option_is_validated(lib):
    o = pmg.pfasst_mg_default_options(slice_groups=9)
    nb = ctypes.c_size_t(0)
    g, fnodes, lv = pmg.pmg_grid(3, 31), pmg.pmg_nodes_desc(5, 0), pmg.pmg_levels(2, pmg.pmg_nodes_desc(3, 0))
    assert lib.pfasst_mg_workspace_bytes(ctypes.byref(g), ctypes.byref(fnodes), ctypes.byref(lv), 8,
                                         ctypes.byref(o), ctypes.byref(nb)) == pmg.PMG_ERR_INVALID_ARG
    sizes = []
    for G in (1, 0, 4):
        o = pmg.pfasst_mg_default_options(slice_groups=G, vcycles=2)
        assert lib.pfasst_mg_workspace_bytes(ctypes.byref(g), ctypes.byref(fnodes), ctypes.byref(lv), 8,
                                             ctypes.byref(o), ctypes.byref(nb)) == pmg.PMG_OK
        sizes.append(nb.value)
    # the pipelined iteration adds a single-grid multigrid scratch for the coarse chain
    assert sizes[0] == sizes[1] < sizes[2]


def test_uniform_node_family_is_accepted_and_checked(lib):
    o = pmg.pfasst_mg_default_options()
    nb = ctypes.c_size_t(0)
    g = pmg.pmg_grid(2, 31)
    ok = lib.pfasst_mg_workspace_bytes(ctypes.byref(g), ctypes.byref(pmg.pmg_nodes_desc(5, 1)),
                                       ctypes.byref(pmg.pmg_levels(2, pmg.pmg_nodes_desc(3, 1))), 4,
                                       ctypes.byref(o), ctypes.byref(nb))
    assert ok == pmg.PMG_OK
    bad = lib.pfasst_mg_workspace_bytes(ctypes.byref(g), ctypes.byref(pmg.pmg_nodes_desc(5, 2)),
                                        ctypes.byref(pmg.pmg_levels(1, pmg.pmg_nodes_desc(0, 0))), 4,
                                        ctypes.byref(o), ctypes.byref(nb))
    assert bad == pmg.PMG_ERR_UNSUPPORTED


def _ws3(lib, g, fnodes, lv, P=4, **kw):
    nb = ctypes.c_size_t(0)
    o = pmg.pfasst_mg_default_options(**kw)
    rc = lib.pfasst_mg_workspace_bytes(ctypes.byref(g), ctypes.byref(fnodes), ctypes.byref(lv), P, ctypes.byref(o),
                                       ctypes.byref(nb))
    return rc, nb.value


def test_three_level_hierarchy_is_validated(lib):
    D = pmg.pmg_nodes_desc
    g = pmg.pmg_grid(3, 31)
    rc2, b2 = _ws3(lib, g, D(5, 0), pmg.pmg_levels(2, D(3, 0)))
    rc3, b3 = _ws3(lib, g, D(5, 0), pmg.pmg_levels(3, D(3, 0), D(2, 0)))
    assert rc2 == rc3 == pmg.PMG_OK and b3 > b2  # level-2 state, its correction and its inverses
    assert _ws3(lib, pmg.pmg_grid(2, 7), D(5, 0), pmg.pmg_levels(3, D(3, 0), D(2, 0)))[0] == pmg.PMG_ERR_INVALID_ARG
    assert _ws3(lib, pmg.pmg_grid(2, 15), D(5, 0), pmg.pmg_levels(3, D(3, 0), D(2, 0)))[0] == pmg.PMG_OK
    assert _ws3(lib, g, D(5, 0), pmg.pmg_levels(3, D(3, 0), D(4, 0)))[0] == pmg.PMG_ERR_INVALID_ARG
    assert _ws3(lib, g, D(5, 0), pmg.pmg_levels(3, D(3, 0), D(1, 0)))[0] == pmg.PMG_ERR_INVALID_ARG
    assert _ws3(lib, g, D(5, 0), pmg.pmg_levels(3, D(3, 0), D(2, 2)))[0] == pmg.PMG_ERR_UNSUPPORTED
    assert _ws3(lib, g, D(5, 0), pmg.pmg_levels(4, D(3, 0), D(2, 0)))[0] == pmg.PMG_ERR_INVALID_ARG
    # with two levels the coarsest description is ignored
    assert _ws3(lib, g, D(5, 0), pmg.pmg_levels(2, D(3, 0), D(7, 5)))[0] == pmg.PMG_OK


def test_create_rejects_coarsest_nodes_that_do_not_nest(lib):
    """Uniform nodes: {0, 1/2, 1} is not a subset of {0, 1/3, 2/3, 1} (which is one of
    {0, 1/6, ..., 1}); the check runs before any device allocation."""
    D = pmg.pmg_nodes_desc
    h = ctypes.c_void_p()
    o = pmg.pfasst_mg_default_options()
    rc = lib.pfasst_mg_create(ctypes.byref(pmg.pmg_grid(1, 63)), ctypes.byref(D(7, 1)),
                              ctypes.byref(pmg.pmg_levels(3, D(4, 1), D(3, 1))), 1.0, 0.01, 2,
                              ctypes.byref(o), None, None, 0, ctypes.byref(h))
    assert rc == pmg.PMG_ERR_INVALID_ARG and not h.value
    assert "coarsest nodes are not a subset" in pmg.pfasst_mg_last_error()


def test_stencil_order_is_validated(lib):
    D = pmg.pmg_nodes_desc
    lv = pmg.pmg_levels(2, D(3, 0))
    for order, n, want in ((0, 31, pmg.PMG_OK), (2, 31, pmg.PMG_OK), (4, 31, pmg.PMG_OK), (4, 7, pmg.PMG_OK),
                           (3, 31, pmg.PMG_ERR_INVALID_ARG), (4, 3, pmg.PMG_ERR_INVALID_ARG)):
        rc, _ = _ws3(lib, pmg.pmg_grid(2, n, order), D(5, 0), lv if n >= 7 else pmg.pmg_levels(1, D(0, 0)))
        assert rc == want, (order, n, rc)
    # the fourth-order fine level needs no extra device memory
    assert _ws3(lib, pmg.pmg_grid(3, 31, 4), D(5, 0), lv)[1] == _ws3(lib, pmg.pmg_grid(3, 31, 2), D(5, 0), lv)[1]
