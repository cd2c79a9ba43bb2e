"""The oracle's pins must catch the mistakes they are meant to catch (CPU only).

Each case copies ``oracle/pic_oracle.c``, plants one plausible slip (a wrong
coefficient in an Esirkepov bracket, the end-point shapes in place of the
path average, a dropped 1/2 or cell volume, gamma in place of gamma - 1),
compiles the copy with gcc into a temporary directory, and runs the pin
against it: the pin has to fail.  The unmodified oracle passes the same pins
in ``test_oracle_pins.py``.  Nothing here touches the GPU path.
"""
import ctypes  # noqa: F401  (the mutant libraries are opened through ctypes)
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "pic_oracle.c")

# (name, original text, planted text, pin that must fail)
MUTANTS = [
    ("2D Jz bracket: 1/3 -> 1/4",
     "DS[0][i] * DS[1][j] / 3.0;", "DS[0][i] * DS[1][j] / 4.0;",
     lambda: pins.check_transverse_moments(2, 2)),
    ("2D Jz from the new shapes alone",
     "double sm = S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] + 0.5 * S0[0][i] * DS[1][j] +",
     "double sm = S1[0][i] * S1[1][j] + 0.0 *",
     lambda: pins.check_transverse_moments(2, 1)),
    ("2D Jz without the x half term",
     "double sm = S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] + 0.5 * S0[0][i] * DS[1][j] +",
     "double sm = S0[0][i] * S0[1][j] + 0.5 * S0[0][i] * DS[1][j] +",
     lambda: pins.check_transverse_moments(2, 2)),
    ("3D Jx bracket: 1/3 -> 1/4",
     "DS[1][j] * DS[2][k] / 3.0);", "DS[1][j] * DS[2][k] / 4.0);",
     lambda: pins.check_transverse_moments(3, 2)),
    ("field energy without the 1/2",
     "ue *= 0.5 * dV;", "ue *= dV;",
     lambda: pins.check_field_energy_of_eigenmode(3)),
    ("magnetic energy without dV",
     "ub *= 0.5 * dV;", "ub *= 0.5;",
     lambda: pins.check_field_energy_of_eigenmode(2)),
    ("kinetic energy without dV",
     "uk += p->w * dV * (gm - sp->m);", "uk += p->w * (gm - sp->m);",
     lambda: pins.check_kinetic_energy_of_cold_beams(3)),
    ("kinetic energy with gamma for gamma - 1",
     "uk += p->w * dV * (gm - sp->m);", "uk += p->w * dV * gm;",
     lambda: pins.check_kinetic_energy_of_cold_beams(2)),
    ("kinetic energy per unit mass",
     "uk += p->w * dV * (gm - sp->m);", "uk += p->w * dV * (gm - sp->m) / sp->m;",
     lambda: pins.check_kinetic_energy_of_cold_beams(2)),
    ("electric energy without the 1/2, seen by the energy exchange",
     "ue *= 0.5 * dV;", "ue *= dV;",
     pins.check_langmuir_energy_exchange),
    ("kinetic energy without dV, seen by the energy exchange",
     "uk += p->w * dV * (gm - sp->m);", "uk += p->w * (gm - sp->m);",
     pins.check_langmuir_energy_exchange),
]


def _compile_mutant(tmp_path, original: str, planted: str) -> str:
    src = open(SRC).read()
    assert src.count(original) == 1, f"the planted site is no longer unique in pic_oracle.c: {original!r}"
    mut = tmp_path / "pic_oracle_mutant.c"
    mut.write_text(src.replace(original, planted))
    lib = tmp_path / "libpic_oracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off", "-o", str(lib), str(mut),
                    "-lm"], check=True)
    return str(lib)


@pytest.mark.parametrize("name,original,planted,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_fails_on_planted_mistake(tmp_path, monkeypatch, name, original, planted, pin):
    lib = oracle.load_library(_compile_mutant(tmp_path, original, planted))
    monkeypatch.setattr(oracle, "_lib", lib)
    with pytest.raises(AssertionError):
        pin()
