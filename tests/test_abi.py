"""The C-ABI library builds, loads and exports every function the header declares (CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sscf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(sscf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sscf_build_fock", "sscf_rotate_sweep", "sscf_orthonormalise", "sscf_density", "sscf_step"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1402_2880_gb300 import _lib, build
    path = build.build()
    assert os.path.exists(path)
    lib = _lib.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(_lib.EXPORTED) == declared_functions()


def test_strerror_without_gpu():
    from paper_1402_2880_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    assert lib.sscf_strerror(0) == b"ok"
    assert lib.sscf_strerror(-5) == b"sparse capacity exceeded"


def test_create_rejects_bad_layout_without_touching_the_gpu():
    import ctypes

    import numpy as np

    from paper_1402_2880_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    species = np.array([1, 0, 1], dtype=np.int32)   # not O, H, H
    xyz = np.zeros(9)
    grp = np.zeros(1, dtype=np.int32)
    sysc = _lib.System(n_atoms=3, species=species.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       xyz=xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       group_of_mol=grp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    from synth import default_params
    prm = _lib.make_params(default_params())
    h = ctypes.c_void_p()
    assert lib.sscf_create(ctypes.byref(sysc), ctypes.byref(prm), None, ctypes.byref(h)) == -1
    with pytest.raises(Exception):
        _lib.Context(species, xyz, grp, default_params())


def test_create_rejects_empty_and_ragged_systems_without_touching_the_gpu():
    """No atoms, a negative count, or a count that is not whole molecules
    (O, H, H) is refused with SSCF_ERR_INVALID_ARG before any CUDA call."""
    import ctypes

    import numpy as np

    from paper_1402_2880_gb300 import _lib, build
    from synth import default_params
    build.build()
    lib = _lib.load()
    prm = _lib.make_params(default_params())
    for n_atoms in (0, -3, 4):
        species = np.tile(np.array([0, 1, 1], dtype=np.int32), 2)
        xyz = np.zeros(18)
        grp = np.zeros(2, dtype=np.int32)
        sysc = _lib.System(n_atoms=n_atoms, species=species.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                           xyz=xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           group_of_mol=grp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        h = ctypes.c_void_p()
        assert lib.sscf_create(ctypes.byref(sysc), ctypes.byref(prm), None, ctypes.byref(h)) == -1
        assert not h.value
