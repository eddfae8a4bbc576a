"""The ctypes structures of the binding have the C layout of include/mpsa.h (CPU only).

A small C program, compiled with the host compiler against the header, prints sizeof and
offsetof of every field; the binding's ctypes structures must agree field by field.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> (binding class name, [(C field, ctypes field)])
PAIRS = {
    "mpsa_elements": ("Elements", ["n_elements", "mass_amu", "chi_eV", "U1", "U2", "log_eps"]),
    "mpsa_lines": ("Lines", ["n_lines", "lambda_nm", "log_gf", "E_eV", "species", "log_gR", "log_gS", "log_gW"]),
    "mpsa_lgrid": ("LGrid", ["lambda0_nm", "lambda1_nm", "R"]),
    "mpsa_synth_opts": ("SynthOpts", ["cut", "kc_factor", "precision", "tile", "continuum", "reserved"]),
    "mpsa_eos": ("Eos", ["n_elements", "mass_amu", "log_eps", "n_stages", "chi_eV", "lnU"]),
    "mpsa_atmos": ("Atmos", ["n_depth", "m", "T", "P", "comp"]),
    "mpsa_odf_table": ("OdfTable", ["nT", "nP", "log10_T", "log10_P", "K", "n_steps", "odf", "kappa_c", "lam_c_nm",
                                    "widths"]),
    "mpsa_batch_group": ("BatchGroup", ["grid", "n_sel", "sel", "kappa_out", "kappa_c_out", "evals_out", "K", "bounds",
                                        "n_steps", "widths", "odf_out", "mean_kind"]),
    "mpsa_batch_info": ("BatchInfo", ["pts_per_thread", "threads", "min_blocks", "n_rows", "n_units", "n_tuned",
                                      "tune_ms_per_mpoint"]),
    "mpsa_request": ("Request", ["kind", "atm", "win", "n_mu", "mu", "I_out", "n_sel", "sel", "grid", "K", "bounds",
                                 "n_steps", "widths", "odf_out", "kappa_c_out", "mean_kind"]),
    "mpsa_server_stats": ("ServerStats", ["submitted", "completed", "failed", "running", "queued", "bytes_in_use",
                                          "bytes_peak"]),
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mpsa.h"', "int main(void) {"]
    for s, (_, fields) in PAIRS.items():
        lines.append(f'    printf("{s} sizeof %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'    printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["    return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for row in out.splitlines():
        s, f, v = row.split()
        layout[(s, f)] = int(v)
    return layout


def test_struct_sizes_and_offsets_match(c_layout):
    from paper_2105_13611_gb300 import binding
    for s, (cls_name, fields) in PAIRS.items():
        cls = getattr(binding, cls_name)
        assert ctypes.sizeof(cls) == c_layout[(s, "sizeof")], (s, ctypes.sizeof(cls), c_layout[(s, "sizeof")])
        assert [f for f, _ in cls._fields_] == fields, (s, [f for f, _ in cls._fields_])
        for f in fields:
            assert getattr(cls, f).offset == c_layout[(s, f)], (s, f, getattr(cls, f).offset, c_layout[(s, f)])
