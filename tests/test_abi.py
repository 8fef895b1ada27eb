"""The C-ABI library loads without a GPU and exports every declared symbol;
host-side MPO construction (no GPU) reproduces the full-CI Hamiltonian."""
import os

import numpy as np
import pytest

import synth
from oracle import fci
from oracle import mps as om

import paper_1902_08489_gb300 as td


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(td.LIB_PATH):
        from paper_1902_08489_gb300 import build
        build.build()
    return td.lib()


def test_exports_every_header_symbol(built):
    syms = td.header_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(built, s)]
    assert not missing, missing
    for s in ["tdmps_build_mpo", "tdmps_mps_from_determinant", "tdmps_apply_H", "tdmps_overlap",
              "tdmps_compress", "tdmps_rk4_step", "tdmps_krylov_step", "tdmps_one_rdm"]:
        assert s in syms


def test_invalid_arguments_are_rejected_without_gpu(built):
    h = np.zeros((2, 2))
    eri = np.zeros((2, 2, 2, 2))
    with pytest.raises(td.TdmpsError) as e:
        td.build_mpo(None, h, eri, L=0)
    assert e.value.name == "INVALID_ARG"
    h[0, 0] = np.nan
    with pytest.raises(td.TdmpsError) as e:
        td.build_mpo(None, h, eri)
    assert e.value.name == "NONFINITE"
    # host-only calls: NULL handles, sites out of range, short buffers
    import ctypes
    assert td.ERRORS[built.tdmps_mps_info(None, None, None, None, None)] == "INVALID_ARG"
    assert td.ERRORS[built.tdmps_mpo_info(None, None, None)] == "INVALID_ARG"
    mpo = td.build_mpo(None, np.diag([-1.0, -0.5]), np.zeros((2, 2, 2, 2)), n_elec=2)
    n = ctypes.c_int64(0)
    for site in (-1, 2):
        assert td.ERRORS[built.tdmps_mpo_elements(mpo.h, site, ctypes.byref(n), None, None, None,
                                                  None, None)] == "INVALID_ARG"
    assert built.tdmps_mpo_elements(mpo.h, 0, ctypes.byref(n), None, None, None, None, None) == 0
    need = n.value
    assert need > 0
    buf = [np.zeros(need, dtype=np.int32) for _ in range(4)]
    vals = np.zeros(need)
    ptrs = [b.ctypes.data_as(ctypes.c_void_p) for b in buf]
    assert td.ERRORS[built.tdmps_mpo_elements(mpo.h, 0, ctypes.byref(n), ptrs[0], None, ptrs[2],
                                              ptrs[3], vals.ctypes.data_as(ctypes.c_void_p))] \
        == "INVALID_ARG"
    short = ctypes.c_int64(need - 1)
    assert td.ERRORS[built.tdmps_mpo_elements(mpo.h, 0, ctypes.byref(short), *ptrs,
                                              vals.ctypes.data_as(ctypes.c_void_p))] == "INVALID_ARG"
    assert short.value == need
    mpo.free()
    # context setters reject a NULL context
    assert td.ERRORS[built.tdmps_set_concurrent_inner(None, 0)] == "INVALID_ARG"
    assert td.ERRORS[built.tdmps_set_krylov_fp64(None, 1)] == "INVALID_ARG"
    # the local operator: a NULL context is refused before anything else,
    # and freeing a NULL operator is a no-op
    assert td.ERRORS[built.tdmps_heff_create(None, mpo.h, None, 0, None, None)] == "INVALID_ARG"
    assert td.ERRORS[built.tdmps_heff_apply(None, None, None, None)] == "INVALID_ARG"
    assert built.tdmps_heff_free(None) == 0


def _dense_mpo(mpo, L):
    """Contract W_0 ... W_{L-1} into the 4^L x 4^L operator (first site
    slowest), from the host copy of the MPO elements."""
    dims, _ = mpo.bond_dims()
    Ws = []
    for i in range(L):
        win, wout, sig, sigp, v = mpo.elements(i)
        W = np.zeros((dims[i], dims[i + 1], 4, 4))
        np.add.at(W, (win, wout, sig, sigp), v)
        Ws.append(W)
    T = Ws[0][0]                       # (w1, 4, 4)
    for i in range(1, L):
        T = np.einsum("wab,wvcd->vacbd", T, Ws[i])
        n = T.shape[1] * T.shape[2]
        T = T.reshape(T.shape[0], n, n)
    assert T.shape[0] == 1
    return T[0]


@pytest.mark.parametrize("L,seed", [(2, 0), (3, 1), (4, 2)])
def test_host_mpo_equals_full_ci_hamiltonian(built, L, seed):
    I = synth.make_integrals(L, seed=seed, n_chol=4)
    mpo = td.build_mpo(None, I.h, I.eri, n_elec=L, e0=0.37)
    Hm = _dense_mpo(mpo, L)
    assert np.abs(Hm - Hm.T).max() < 1e-12
    for na in range(L + 1):
        for nb in range(L + 1):
            dets = fci.basis(L, na, nb)
            idx = om.fock_index(dets, L)
            ref = fci.hamiltonian(I.h, I.eri, dets, e0=0.37)
            assert np.allclose(Hm[np.ix_(idx, idx)], ref, atol=1e-12)
    # no matrix elements between different (N, S_z) sectors
    blocks = np.zeros_like(Hm)
    for na in range(L + 1):
        for nb in range(L + 1):
            idx = om.fock_index(fci.basis(L, na, nb), L)
            blocks[np.ix_(idx, idx)] = Hm[np.ix_(idx, idx)]
    assert np.abs(Hm - blocks).max() == 0.0


def test_mpo_bond_dimension_is_quadratic_in_the_smaller_side(built):
    L = 16
    I = synth.make_integrals(L, seed=0)
    mpo = td.build_mpo(None, I.h, I.eri, n_elec=16)
    dims, nel = mpo.bond_dims()
    assert dims[0] == 1 and dims[L] == 1
    # complementary-operator count: 2 + 4L singles + O(8 min(k, L-k)^2) pairs
    for k in range(1, L):
        m = min(k, L - k)
        assert dims[k] <= 2 + 4 * L + 8 * m * m + 8 * m, (k, dims[k])
    assert dims[L // 2] <= 600


def test_binding_constants_match_the_header():
    """The Python binding's precision codes, error codes and statistics
    classes equal the enums of include/tdmps.h."""
    import re
    src = open(os.path.join(os.path.dirname(td.__file__), "..", "include", "tdmps.h")).read()
    enum = {m.group(1): int(m.group(2))
            for m in re.finditer(r"\bTDMPS_([A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    for name, code in td.PRECISION.items():
        assert enum[name.upper()] == code
    for code, name in td.ERRORS.items():
        assert enum["ERR_" + name] == code
    assert {k for k in enum if k.startswith("ERR_")} == {"ERR_" + n for n in td.ERRORS.values()}
    for name, k in td.KSTAT.items():
        assert enum["KSTAT_" + name.upper()] == k
    assert enum["KSTAT_COUNT"] == len(td.KSTAT)


def test_binding_signatures_match_the_header_prototypes():
    """Every entry point of include/tdmps.h has a ctypes signature in the
    binding with the same number of arguments and the same kind of each
    (pointer or handle, int, int64, double, complex by value)."""
    import ctypes
    import re
    src = open(os.path.join(os.path.dirname(td.__file__), "..", "include", "tdmps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = {m.group(2): (m.group(1), m.group(3)) for m in re.finditer(
        r"^\s*(int|const char\*)\s+(tdmps_\w+)\(([^;]*?)\);", src, re.M | re.S)}
    assert set(protos) == set(td.header_symbols())

    def kind_c(p):
        p = " ".join(p.split())
        if "*" in p or re.search(r"\btdmps_(ctx|mpo|mps|heff)_t\b", p):
            return "ptr"
        if re.search(r"\btdmps_complex\b", p):
            return "complex"
        if "int64_t" in p:
            return "int64"
        if re.search(r"\bdouble\b", p):
            return "double"
        if re.search(r"\bint\b", p):
            return "int"
        raise AssertionError(p)

    def kind_py(t):
        if t is ctypes.c_void_p or t is ctypes.c_char_p or hasattr(t, "_type_") and \
                issubclass(t, ctypes._Pointer):
            return "ptr"
        return {ctypes.c_int: "int", ctypes.c_int64: "int64", ctypes.c_double: "double",
                td.Complex: "complex"}[t]

    for name, (ret, params) in protos.items():
        assert name in td._SIGS, name
        restype, argtypes = td._SIGS[name]
        assert restype is (ctypes.c_int if ret == "int" else ctypes.c_char_p), name
        plist = [p for p in params.split(",") if p.strip() and p.strip() != "void"]
        assert [kind_c(p) for p in plist] == [kind_py(t) for t in argtypes], name


def test_binding_structs_match_the_header():
    """tdmps_complex and tdmps_kstat: same fields, order and types as the
    ctypes mirrors Complex and KStat."""
    import ctypes
    import re
    src = open(os.path.join(os.path.dirname(td.__file__), "..", "include", "tdmps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    ctype = {"double": ctypes.c_double, "int64_t": ctypes.c_int64, "int": ctypes.c_int}
    for cname, mirror in (("tdmps_complex", td.Complex), ("tdmps_kstat", td.KStat)):
        body = re.search(r"typedef struct \{([^}]*)\}\s*%s;" % cname, src).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            typ, names = decl.split(None, 1)
            fields += [(n.strip(), ctype[typ]) for n in names.split(",")]
        assert fields == list(mirror._fields_), cname
