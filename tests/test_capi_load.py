"""The C-ABI library loads and exports every symbol include/*.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names.update(re.findall(r"JMD_API\s+[\w\s\*]*?\b(md_\w+)\s*\(", txt))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for n in ("md_space_periodic", "md_nbr_plan", "md_neighbor_list_build", "md_neighbor_list_update",
              "md_energy_forces", "md_integrate_nve", "md_minimize", "md_status_poll"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import importlib.util
    spec = importlib.util.spec_from_file_location("_jmd_build", os.path.join(ROOT, "paper_1912_04232_b300", "build.py"))
    build = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(build)
    lib = ctypes.CDLL(build.build())
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_1912_04232_b300 as P
    missing = [n for n in sorted(_declared()) if not hasattr(P, n)]
    assert not missing, missing


def test_binding_loads_and_host_validation():
    import paper_1912_04232_b300 as P
    assert "sm_103a" in P.md_version()
    s = P.md_space_periodic(3, [10.0, 10.0, 10.0])
    assert abs(s.L[0] - 10.0) < 1e-6 and abs(s.Linv[0] - 0.1) < 1e-7
    with pytest.raises(P.MDError) as e:
        P.md_nbr_plan(s, 100, 2.5, 2.6, 64)      # r_list 5.1 > L/2
    assert e.value.code == P.MD_ERR_BOX_TOO_SMALL
    nb = P.md_nbr_plan(s, 100, 2.5, 0.3, 64)
    assert list(nb.ncell) == [3, 3, 3] and nb.ws_bytes > 0
    with pytest.raises(P.MDError):
        P.md_space_periodic(4, [1.0] * 4)
    with pytest.raises(P.MDError):
        P.md_nbr_plan(s, 100, 2.5, 0.3, 1024)     # cap above the supported 512
    for n in (0, -5):                             # empty and negative systems
        with pytest.raises(P.MDError) as e:
            P.md_nbr_plan(s, n, 2.5, 0.3, 64)
        assert e.value.code == P.MD_ERR_INVALID
