"""The C ABI library builds, loads without a GPU and exports every entry
point that include/stmf.h declares; host-side logic of the binding."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "stmf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stmf_[a-z_0-9A-Z]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("stmf_maxplus", "stmf_update_U", "stmf_update_V", "stmf_factorize",
                     "stmf_problem_create", "stmf_create", "stmf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2205_06619_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_export_list_matches_header():
    from paper_2205_06619_gb300 import api
    assert sorted(api.EXPORTS) == sorted(n for n in declared_functions())


def test_default_options_without_gpu():
    from paper_2205_06619_gb300 import api
    lib = api.load()
    o = api.Options()
    lib.stmf_default_options(ctypes.byref(o))
    assert o.sweeps == 1 and o.acol_p == 5 and o.window == 0 and o.seed == 0 and not o.trace and not o.mlp
    # the evaluation's launch shapes default to the library's choice
    assert (o.res_chunk, o.delta_blocks_per_sm, o.delta_tile_rows) == (0, 0, 0)


def test_struct_layouts_match_the_library():
    """The binding's ctypes structs have the sizes the library was built with."""
    from paper_2205_06619_gb300 import api
    lib = api.load()
    sizes = [ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()]
    lib.stmf_struct_sizes(*[ctypes.byref(x) for x in sizes])
    assert [x.value for x in sizes] == [ctypes.sizeof(api.Options), ctypes.sizeof(api.Report),
                                        ctypes.sizeof(api.BatchProblem)]


def test_selection_names_match_the_header():
    """The binding's selection names carry the values of stmf.h's STMF_SEL_*
    (Section "The ByRow strategy"), the default is TD_A, and unknown names are
    refused before any call."""
    from paper_2205_06619_gb300 import api
    text = open(os.path.join(ROOT, "include", "stmf.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"STMF_SEL_([A-Z_]+)\s*=\s*(\d+)", text))
    assert enum == api.SELECTIONS
    o = api.Options()
    api.load().stmf_default_options(ctypes.byref(o))
    assert o.selection == api.SELECTIONS["TD_A"]
    with pytest.raises(ValueError):
        api._selection("BEST")
    strategies = dict((k, int(v)) for k, v in re.findall(r"STMF_STRATEGY_([A-Z_]+)\s*=\s*(\d+)", text))
    assert {k.upper(): v for k, v in api.STRATEGIES.items()} == strategies
    assert o.strategy == api.STRATEGIES["ByRow"]
    with pytest.raises(ValueError):
        api._strategy("ByColumn")


def test_invalid_arguments_fail_without_launch():
    """A NULL context and bad sizes are rejected on the host (no GPU needed)."""
    from paper_2205_06619_gb300 import api
    lib = api.load()
    st = lib.stmf_maxplus(None, 0, 4, 2, None, 2, None, 4, None, 0, None, 4, None, 4, None)
    assert st == 1


def test_mask_packing_layout():
    """Bit t%32 of word t/32 of row s <=> entry (s, t) given (include/stmf.h)."""
    torch = pytest.importorskip("torch")
    from paper_2205_06619_gb300 import api
    rng = np.random.default_rng(0)
    M = rng.random((5, 70)) < 0.5
    # packing runs on the host; only the final .cuda() needs a GPU
    if not torch.cuda.is_available():
        orig = torch.Tensor.cuda
        torch.Tensor.cuda = lambda self, *a, **k: self
        try:
            api_torch = api._torch
            api._torch = lambda: torch
            W = api.pack_mask(M).numpy().view(np.uint32)
        finally:
            torch.Tensor.cuda = orig
            api._torch = api_torch
    else:
        W = api.pack_mask(M).cpu().numpy().view(np.uint32)
    assert W.shape == (5, 3)
    for s in range(5):
        for t in range(70):
            assert bool((W[s, t // 32] >> (t % 32)) & 1) == M[s, t]


def test_sweep_log_summarises_trace_records():
    from paper_2205_06619_gb300 import api
    trace = [(0, 3, 2, 7, 1, 0, 10.0), (0, 1, -1, -1, -1, -1, 10.0), (0, 0, 4, 2, 0, 1, 8.5),
             (1, 3, -1, -1, -1, -1, 8.5), (1, 1, 0, 5, 1, 0, 8.0), (1, 0, -1, -1, -1, -1, 8.0)]
    log = api.sweep_log(trace)
    assert log == [{"sweep": 0, "rows": 3, "accepted": 2, "f": 8.5, "mean_kept_position": 3.0},
                   {"sweep": 1, "rows": 3, "accepted": 1, "f": 8.0, "mean_kept_position": 0.0}]
    # ByElement records: kept updates at element positions, then the sweep's end record
    trace = [(0, 0, 3, 3, 1, 0, 9.0), (0, 2, 17, 1, 0, 1, 7.0), (0, -1, -1, -1, -1, -1, 7.0),
             (1, -1, -1, -1, -1, -1, 7.0)]
    assert api.sweep_log(trace) == [{"sweep": 0, "rows": 3, "accepted": 2, "f": 7.0, "mean_kept_position": 10.0},
                                    {"sweep": 1, "rows": 1, "accepted": 0, "f": 7.0, "mean_kept_position": None}]


def test_options_carry_selection_and_strategy():
    """The binding writes the selection and strategy into the fields the
    library reads (host-only: the struct is filled, nothing is launched)."""
    from paper_2205_06619_gb300 import api
    o, _ = api._options(3, selection="TD", strategy="ByElement")
    assert (o.sweeps, o.selection, o.strategy) == (3, api.SELECTIONS["TD"], api.STRATEGIES["ByElement"])
    o, _ = api._options(1, strategy="ByMatrix")
    assert (o.selection, o.strategy) == (api.SELECTIONS["TD_A"], api.STRATEGIES["ByMatrix"])
    # the two fields sit at the end of the C struct, after the MLP handle
    assert api.Options.strategy.offset > api.Options.selection.offset > api.Options.mlp.offset
    # launch shapes: (res_chunk, delta_blocks_per_sm[, delta_tile_rows])
    o, _ = api._options(1, shapes=(72, 3, 8))
    assert (o.res_chunk, o.delta_blocks_per_sm, o.delta_tile_rows) == (72, 3, 8)
    o, _ = api._options(1, shapes=(40, 4))
    assert (o.res_chunk, o.delta_blocks_per_sm, o.delta_tile_rows) == (40, 4, 0)
