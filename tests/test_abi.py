"""The C-ABI library builds for sm_103a, loads, exports every function the
public header declares, and its structs have the layout the binding uses.
No compute call is made (no GPU is needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2605_14526_b300 import binding
from paper_2605_14526_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pd_b300.h")


@pytest.fixture(scope="module")
def lib():
    build()
    return ctypes.CDLL(binding.LIB_PATH)


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pd_create" in names and "pd_backward" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    L = binding.lib()
    for n in _declared():
        # the binding declares an argument list for every function of the header
        assert getattr(L, n).argtypes is not None, n


def test_binding_constants_equal_header_enums():
    """Every PD_* enumerator of the header that the binding names has the
    header's value (the model ids, trust-region and solve modes, L-BFGS
    tasks)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"(PD_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            vals[name] = int(val)
    assert vals["PD_COROT_LOGVOL"] == 3
    named = [n for n in vals if hasattr(binding, n)]
    assert {"PD_COROTATED", "PD_NEOHOOKEAN", "PD_COROT_VOLUME", "PD_COROT_LOGVOL"} <= set(named)
    for n in named:
        assert getattr(binding, n) == vals[n], n
    assert sorted(binding.MODELS.values()) == [0, 1, 2, 3]


def test_default_options_and_version(lib):
    o = binding.pd_default_options()
    assert o.aa_m == 5 and o.k_max == 200 and o.local_fp32 == 1
    assert abs(o.eps_tr - 0.1) < 1e-15 and abs(o.eps_step - 1e-8) < 1e-20
    assert "sm_103a" in binding.pd_version()


def test_struct_layouts_match_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "pd_b300.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(pd_mesh), sizeof(pd_material), sizeof(pd_options), sizeof(pd_stats),
         sizeof(pd_profile_out));
  printf("%zu %zu %zu %zu\\n", offsetof(pd_material, gravity), offsetof(pd_options, eps_step),
         offsetof(pd_stats, factor_nnz), offsetof(pd_stats, last_rho));
  printf("%zu %zu\\n", sizeof(pd_lbfgs_options), offsetof(pd_lbfgs_options, gtol));
  printf("%zu %zu %zu\\n", sizeof(pd_contact_desc), offsetof(pd_contact_desc, attach_target),
         offsetof(pd_contact_desc, attach_steps));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[:5] == [ctypes.sizeof(binding.pd_mesh), ctypes.sizeof(binding.pd_material),
                         ctypes.sizeof(binding.pd_options), ctypes.sizeof(binding.pd_stats),
                         ctypes.sizeof(binding.pd_profile_out)]
    assert sizes[5:9] == [binding.pd_material.gravity.offset, binding.pd_options.eps_step.offset,
                          binding.pd_stats.factor_nnz.offset, binding.pd_stats.last_rho.offset]
    assert sizes[9:11] == [ctypes.sizeof(binding.pd_lbfgs_options), binding.pd_lbfgs_options.gtol.offset]
    assert sizes[11:] == [ctypes.sizeof(binding.pd_contact_desc), binding.pd_contact_desc.attach_target.offset,
                          binding.pd_contact_desc.attach_steps.offset]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        binding.lib()
