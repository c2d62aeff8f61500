"""The C-ABI library loads on a machine without a GPU and exports every symbol
``include/lbm_mix.h`` declares; the ctypes mirror of ``lbm_mix_params``
matches the C layout; argument validation fails cleanly before any CUDA call."""

import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_mix.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"LBM_API\s+[\w\s\*]+?\b(lbm_mix_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["lbm_mix_create", "lbm_mix_init_fields", "lbm_mix_step", "lbm_mix_get_moments",
                     "lbm_mix_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(built_library):
    lib = ct.CDLL(str(built_library))
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", str(built_library)], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(lbm_mix_\w+)\b", out))
    assert exported == set(_declared())


def test_binding_mirrors_header(built_library):
    from paper_2004_11286_gb300 import binding
    assert set(binding.SIGNATURES) == set(_declared())
    lib = binding.load_library()
    assert lib.lbm_mix_num_outputs(3) == 6 + 5 * 3


def test_params_struct_layout(tmp_path):
    from paper_2004_11286_gb300.binding import lbm_mix_params
    c = tmp_path / "layout.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm_mix.h"\n'
                 "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(lbm_mix_params),"
                 " offsetof(lbm_mix_params, omega_fixed), offsetof(lbm_mix_params, nx),"
                 " offsetof(lbm_mix_params, slaved_species), offsetof(lbm_mix_params, fp64_cond_bound),"
                 " offsetof(lbm_mix_params, closure_residual_bound), offsetof(lbm_mix_params, cv_terms),"
                 " offsetof(lbm_mix_params, jet_X), offsetof(lbm_mix_params, jet_P),"
                 " offsetof(lbm_mix_params, jet_y1));"
                 "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    P = lbm_mix_params
    assert vals == [ct.sizeof(P), P.omega_fixed.offset, P.nx.offset, P.slaved_species.offset,
                    P.fp64_cond_bound.offset, P.closure_residual_bound.offset, P.cv_terms.offset,
                    P.jet_X.offset, P.jet_P.offset, P.jet_y1.offset]


def _params(M=2, **over):
    from paper_2004_11286_gb300.binding import lbm_mix_params, _DP
    import numpy as np
    keep = [np.array([4.0, 40.0][:M]), np.array([1.5, 1.5][:M]), np.array([[0, .05], [.05, 0]])[:M, :M].ravel().copy(),
            np.array([0.003, 0.003][:M]), np.array([0.01, 0.01][:M])]
    p = lbm_mix_params()
    p.M = M
    p.molar_mass, p.cv_molar, p.D, p.mu, p.lambda_ = (a.ctypes.data_as(_DP) for a in keep)
    p.R_U, p.nx, p.ny, p.nz = 1.0, 8, 8, 8
    p.slaved_species, p.precision, p.coupling, p.closure = -1, 1, 0, 0
    for k, v in over.items():
        setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("field,value,status", [
    ("M", 0, 1), ("M", 9, 1), ("nx", 0, 1), ("R_U", 0.0, 1), ("precision", 7, 1),
    ("coupling", 5, 1), ("closure", 3, 1), ("slaved_species", 4, 1),
])
def test_create_rejects_bad_arguments_without_touching_cuda(built_library, field, value, status):
    from paper_2004_11286_gb300 import binding
    lib = binding.load_library()
    p, keep = _params(**{field: value})
    h = ct.c_void_p()
    st = lib.lbm_mix_create(ct.byref(p), None, ct.byref(h))
    assert st == status
    assert h.value is None
    assert lib.lbm_mix_last_error(None).decode()


def test_create_rejects_grids_of_2_31_nodes(built_library):
    # neighbour indices are 32-bit: 2^31 nodes and more are refused up front
    from paper_2004_11286_gb300 import binding
    lib = binding.load_library()
    p, keep = _params(nx=2048, ny=1024, nz=1024)
    h = ct.c_void_p()
    assert lib.lbm_mix_create(ct.byref(p), None, ct.byref(h)) == 1
    assert h.value is None
    assert b"2^31" in lib.lbm_mix_last_error(None)


def test_closure_network_only_in_fp32_arithmetic(built_library):
    # the learned closure runs in the FP32-arithmetic precisions with M >= 2
    from paper_2004_11286_gb300 import binding
    lib = binding.load_library()
    p, keep = _params(precision=0, closure=1)
    h = ct.c_void_p()
    assert lib.lbm_mix_create(ct.byref(p), None, ct.byref(h)) == 2
    assert h.value is None


def test_closure_sizes_match_the_oracle(built_library):
    from paper_2004_11286_gb300 import binding
    from oracle import closure as CL
    for M in range(1, 9):
        F, O, nw = binding.closure_sizes(M)
        assert (F, O) == CL.closure_dims(M)[:2]
        assert nw == CL.weight_count(M)
    with pytest.raises(binding.LbmError):
        binding.closure_sizes(9)


@pytest.mark.parametrize("bc,status", [
    ([1, 0, 0, 0, 0, 0], 2),      # a wall on one x face only
    ([0, 0, 1, 1, 0, 0], 2),      # walls normal to y
    ([1, 1, 1, 1, 0, 0], 2),
    ([7, 7, 0, 0, 0, 0], 1),      # unknown boundary type
])
def test_create_rejects_unbuilt_boundaries(built_library, bc, status):
    from paper_2004_11286_gb300 import binding
    lib = binding.load_library()
    p, keep = _params()
    for k in range(6):
        p.bc[k] = bc[k]
    h = ct.c_void_p()
    assert lib.lbm_mix_create(ct.byref(p), None, ct.byref(h)) == status
    assert h.value is None


def test_walls_with_the_network_closure_are_refused(built_library):
    from paper_2004_11286_gb300 import binding
    lib = binding.load_library()
    p, keep = _params(closure=1)
    p.bc[0] = p.bc[1] = 1
    h = ct.c_void_p()
    assert lib.lbm_mix_create(ct.byref(p), None, ct.byref(h)) == 2
    assert b"periodic" in lib.lbm_mix_last_error(None)


def test_create_rejects_nonperiodic_and_asymmetric(built_library):
    from paper_2004_11286_gb300 import binding
    import numpy as np
    lib = binding.load_library()
    p, keep = _params()
    p.bc[1] = 1
    h = ct.c_void_p()
    assert lib.lbm_mix_create(ct.byref(p), None, ct.byref(h)) == 2
    p, keep = _params()
    bad = np.array([0, .05, .06, 0.0])
    p.D = bad.ctypes.data_as(binding._DP)
    assert lib.lbm_mix_create(ct.byref(p), None, ct.byref(h)) == 1
    assert "symmetric" in lib.lbm_mix_last_error(None).decode()


def test_null_handle_calls_fail_cleanly(built_library):
    from paper_2004_11286_gb300 import binding
    lib = binding.load_library()
    assert lib.lbm_mix_step(None, 1) == 1
    assert lib.lbm_mix_destroy(None) == 1
    assert lib.lbm_mix_step_count(None) == -1


def test_make_params_jets():
    """The opposed-jets boundary set through the binding: jet faces on x,
    outlets on y, z periodic, and the nozzle and inlet fields as given."""
    import types
    import numpy as np
    from paper_2004_11286_gb300 import binding
    jets = types.SimpleNamespace(y0=3, y1=9, X=np.array([[0.2, 0.8], [0.6, 0.4]]), u=np.array([0.01, -0.02]),
                                 T=np.array([0.2, 0.3]), P=np.array([0.01, 0.02]))
    p, keep = binding.make_params([2.0, 28.0], [2.5, 2.5], [[0, 0.05], [0.05, 0]], mu=[0.1, 0.1], lam=[0.1, 0.1],
                                  shape=(1, 12, 10), jets=jets)
    assert list(p.bc) == [2, 2, 3, 3, 0, 0]
    assert (p.jet_y0, p.jet_y1) == (3, 9)
    assert [p.jet_X[k] for k in range(4)] == [0.2, 0.8, 0.6, 0.4]
    assert list(p.jet_u) == [0.01, -0.02] and list(p.jet_T) == [0.2, 0.3] and list(p.jet_P) == [0.01, 0.02]
    p2, _ = binding.make_params([2.0, 28.0], [2.5, 2.5], [[0, 0.05], [0.05, 0]], mu=[0.1, 0.1], lam=[0.1, 0.1])
    assert list(p2.bc) == [0] * 6 and not p2.jet_X
