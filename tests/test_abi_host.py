"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports
every function include/emu.h declares, and its host-only logic (configuration
validation, workspace sizing) behaves.  No call here touches a GPU."""
import re
from pathlib import Path

import pytest

from paper_2101_02745_gb300 import build as B
from paper_2101_02745_gb300 import emu as E

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    B.build()
    return E.load()


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(emu_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("emu_create", "emu_bind", "emu_init_particles", "emu_deposit", "emu_interpolate_H",
                     "emu_rk_stage", "emu_step", "emu_moments", "emu_timestep", "emu_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_has_no_cpu_fallback_symbols(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", str(B.LIB)], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert {n for n in exported if n.startswith("emu_")} == set(declared_functions())
    assert not any(n.startswith("or_") for n in exported)


def test_workspace_and_config_validation(lib):
    cfg = E.make_config(32, 16, 13.42, 1.9e-22, 3e10)
    n1 = E.emu_workspace_bytes(cfg)
    assert n1 > 0 and n1 % 256 == 0
    big = E.make_config(16384, 1000, 1024.0, 1.9e-22, 3e10)
    assert E.emu_workspace_bytes(big) > n1
    for bad in (E.make_config(0, 16, 1.0, 1e-22, 3e10), E.make_config(4, 0, 1.0, 1e-22, 3e10),
                E.make_config(4, 4, -1.0, 1e-22, 3e10), E.make_config(4, 4, 1.0, 1e-22, 3e10, shape_order=4),
                E.make_config(4, 4, 1.0, 1e-22, 3e10, shape_order=-1)):
        with pytest.raises(E.EmuError) as ei:
            E.emu_create(bad)
        assert ei.value.code == E.EMU_EINVAL
        assert E.emu_workspace_bytes.__name__  # message is set
        assert E.emu_last_error(None)


def test_oversized_box_rejected(lib):
    """A box whose units (tiles x directions) overflow the kernels' int index is rejected."""
    cfg = E.make_config(30 * 40000, 60000, 1.0e5, 1.9e-22, 3e10)   # 40000 tiles x 60000 directions > 2^31
    assert E.load().emu_workspace_bytes(cfg) == E.EMU_EINVAL


def test_shape_orders_geometry(lib):
    """Orders 0-2 tile 30 cells per warp, order 3 (two halo lanes a side) 28;
    the kept shape weights: none (order 0), 3 (1, 2) or 5 (3) per particle."""
    sizes = {o: E.emu_workspace_bytes(E.make_config(840, 10, 52.5, 1.9e-22, 3e10, shape_order=o)) for o in range(4)}
    for o in range(4):
        box = E.emu_create(E.make_config(840, 10, 52.5, 1.9e-22, 3e10, shape_order=o))
        E.emu_destroy(box)
    P = 8400
    assert sizes[1] == sizes[2]
    assert sizes[1] - sizes[0] >= 3 * 8 * P - 256
    assert sizes[3] - sizes[2] >= 2 * 8 * P - 256
    mixed = [E.make_config(20, 4, 1.0, 1.9e-22, 3e10, shape_order=1), E.make_config(20, 4, 1.0, 1.9e-22, 3e10)]
    _, ptr = E._cfg_array(mixed)
    assert E.load().emu_batch_workspace_bytes(ptr, 2) == E.EMU_EINVAL


def test_create_destroy_and_unbound_calls(lib):
    cfg = E.make_config(8, 4, 1.0, 1.9e-22, 3e10)
    box = E.emu_create(cfg)
    with pytest.raises(E.EmuError) as ei:
        E.emu_step(box, 1, 1e-12)
    assert ei.value.code == E.EMU_EINVAL and "bind" in str(ei.value)
    assert E.emu_kernel_launches(box) == 0
    E.emu_destroy(box)


def test_oracle_builds_and_is_separate():
    from oracle import oracle as O
    O.build()
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", str(O._LIB)], capture_output=True, text=True).stdout
    assert "or_rk4_step" in out and "emu_step" not in out


def test_autotune_candidate_table_matches_the_header():
    """The binding's table of autotuner candidates (used to put a twin box in
    the configuration the autotuner chose) against the list in include/emu.h:
    its count and, per candidate, the step form, grid, RK form and deposit form."""
    text = (ROOT / "include" / "emu.h").read_text()
    assert int(re.search(r"#define EMU_AUTOTUNE_CANDIDATES (\d+)", text).group(1)) == E.AUTOTUNE_CANDIDATES
    expect = []
    for c in range(E.AUTOTUNE_CANDIDATES):
        if c < 6:
            expect.append((0, (304, 152, 608)[c // 2], c % 2, 0))
        elif c < 10:
            expect.append((1, (304, 152)[(c - 6) // 2], c % 2, 0))
        elif c < 13:
            expect.append((2, (304, 152, 608)[c - 10], -1, 0))
        else:
            expect.append((0, 304, c % 2, 1 if c < 15 else 2))
    assert list(E.AUTOTUNE_GRID_FORMS) == expect
