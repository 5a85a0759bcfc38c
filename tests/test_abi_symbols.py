"""The C-ABI library builds, loads and exports every entry point include/sedacs.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "sedacs.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(sedacs_[a-z0-9_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    from paper_2606_03140_gb300 import build as b

    lib = b.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (sedacs_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_loads_and_names_match_the_header():
    from paper_2606_03140_gb300 import sedacs as S

    for name in _declared():
        assert hasattr(S._lib, name)
    assert set(S.EXPORTED) <= set(_declared())
    p = S.sedacs_default_params()
    assert p.core_size == 32 and p.precision == 1 and abs(p.tau - 1e-3) < 1e-15


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    from paper_2606_03140_gb300 import inputs as I
    from paper_2606_03140_gb300 import sedacs as S

    with pytest.raises(S.SedacsError):
        S.sedacs_create([0, 7, 2], [20.0, 20.0, 20.0], I.SKModel(), S.sedacs_default_params())   # bad species
    with pytest.raises(S.SedacsError):
        S.sedacs_create([0, 0], [4.0, 20.0, 20.0], I.SKModel(), S.sedacs_default_params())      # box < r_off
