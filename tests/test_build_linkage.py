"""The four storage precisions are compiled from one source with a macro
(lb_prec_impl.cuh).  Any helper whose body depends on that macro but whose
symbol does not carry the precision would be emitted under the same name by
all four objects, and the linker would keep one body for all precisions (a
FP64 context launching the FP32 kernel).  This test fails if two precision
objects define the same global or weak symbol."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUILD = os.path.join(ROOT, "paper_1405_2232_gb300", "_build")
ALLOWED = {"DW.ref.__gxx_personality_v0"}


def test_no_symbol_shared_between_precision_objects():
    from paper_1405_2232_gb300 import build
    build.build()
    objs = sorted(f for f in os.listdir(BUILD) if f.startswith("lb_prec_") and f.endswith(".o"))
    assert len(objs) == 4
    seen = {}
    for o in objs:
        try:
            out = subprocess.run(["nm", "--defined-only", os.path.join(BUILD, o)],
                                 capture_output=True, text=True, check=True).stdout
        except FileNotFoundError:
            pytest.skip("nm not available")
        for line in out.splitlines():
            parts = line.split()
            if len(parts) == 3 and parts[1] in "WTVuBDR":
                seen.setdefault(parts[2], set()).add(o)
    shared = {s: sorted(v) for s, v in seen.items() if len(v) > 1 and s not in ALLOWED}
    assert not shared, f"symbols defined by several precision objects: {list(shared)[:5]}"


def test_every_strip_kernel_width_is_compiled():
    """The strip kernel exists at width 128 for every precision and at 256 for the
    FP32 and 16-bit modes (the launcher returns cudaErrorInvalidValue otherwise);
    the 16-bit modes use their own strip kernel, k_step_strip_dev."""
    from paper_1405_2232_gb300 import build
    build.build()
    want = {"fp64": ["128"], "fp32": ["128", "256"], "fp16": ["128", "256"], "bf16": ["128", "256"]}
    prec_id = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
    for name, widths in want.items():
        out = subprocess.run(["nm", "--defined-only", os.path.join(BUILD, f"lb_prec_{name}.o")],
                             capture_output=True, text=True, check=True).stdout
        for w in widths:
            kern = "k_step_strip_dev" if name in ("fp16", "bf16") else "k_step_strip"
            tag = f"{kern}ILi{prec_id[name]}ELi{w}E"
            assert tag in out, f"{name}: no strip kernel of width {w}"
