"""Source check (no GPU) of the known-zero tile flags' invariant.

The stepping launches skip a dry tile whose output buffer already holds the
zero state, which they know from per-tile flags.  The flags describe the
buffers only while the stepping launches are their sole writer, so every
C-ABI call that takes a simulation must do one of three things:
- step it through run_steps;
- only read it;
- clear the flags when it returns (a `ZkReset` declared first).

Two more lists: calls that write only the control block (the owned rows and
the CFL maximum of a strip), and the row exchange of a decomposed domain,
which updates the flags (and the mass bits) of exactly the tiles it writes.

This test holds every such call of the library's sources to one of those
lists.  A new call must be placed in one before the suite passes again.
Ensemble steps must clear the flags of every member.
"""
import pathlib
import re

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2104_06784_gb300" / "csrc"

STEPPING = {"moses_step", "moses_step_timed", "moses_step_dt", "moses_run_until"}
READ_ONLY = {"moses_next_dt", "moses_max_speed", "moses_get_conserved_device", "moses_get_conserved",
             "moses_get_state", "moses_get_budget", "moses_destroy", "moses_get_rows_device"}
CONTROL_ONLY = {"moses_set_owned_rows", "moses_set_max_speed"}
KEEPS_FLAGS = {"moses_set_rows_device"}


def _bodies():
    """name -> body of every `int|void moses_*(moses_sim *s, ...)` definition."""
    out = {}
    for f in sorted(SRC.glob("*.cu")):
        text = f.read_text()
        for m in re.finditer(r"^(?:int|void) (moses_\w+)\(moses_sim \*s\b[^;{]*\{", text, re.M):
            depth, k = 1, m.end()
            while depth:
                depth += {"{": 1, "}": -1}.get(text[k], 0)
                k += 1
            out[m.group(1)] = text[m.end():k - 1]
    return out


def test_every_call_on_a_simulation_keeps_the_flags_valid():
    bodies = _bodies()
    assert "moses_set_conserved" in bodies and "moses_step" in bodies and "moses_adjoint_misfit" in bodies
    for name, body in bodies.items():
        if name in STEPPING:
            assert "run_steps(" in body, name
            assert "ZkReset" not in body, name
        elif name in READ_ONLY:
            assert "ZkReset" not in body, name
        elif name in CONTROL_ONLY:
            assert "ZkReset" not in body, name
            assert "unpack_kernel" not in body, name
            assert all("cudaMemcpyAsync(&s->ctl->amax," in ln for ln in body.splitlines() if "Memcpy" in ln), name
        elif name in KEEPS_FLAGS:
            assert "ZkReset" not in body, name
            assert "rows_replaced<" in body, name
        else:
            first = body.strip().splitlines()[0].strip()
            assert first == "const ZkReset zr{s};", f"{name}: declare `const ZkReset zr{{s}};` first, or list it"


def test_ensemble_steps_clear_the_members_flags():
    text = (SRC / "moses.cu").read_text()
    m = re.search(r"^static int batch_step\(moses_batch \*b, int nsteps, double \*ms\)\n\{", text, re.M)
    assert m is not None
    body = text[m.end():m.end() + 600]
    assert "for (moses_sim *m : b->sims) zk_reset(m);" in body


def test_stepping_sets_the_flags_valid_only_after_its_launches():
    text = (SRC / "moses.cu").read_text()
    start = text.index("static int launch_steps(")
    body = text[start:text.index("\nstatic int set_mode(", start)]
    first_false = body.index("s->zk_valid = false;")
    assert first_false < body.index("launch_stage<T>(")
    # every `zk_valid = zk_on` comes after the last stage launch of its branch
    for m in re.finditer(r"s->zk_valid = zk_on;", body):
        assert body.rfind("launch_stage<T>(", 0, m.start()) > first_false


def test_row_exchange_updates_the_flags_of_the_tiles_it_writes():
    text = (SRC / "moses.cu").read_text()
    start = text.index("int rows_replaced(moses_sim *s, int j0, int j1)")
    body = text[start:text.index("\n}\n", start)]
    assert "fill_ghosts_rows_kernel" in body  # the ghosts those rows own
    assert "cudaMemsetAsync(s->zk + (size_t)ty0 * gx, 0, (size_t)(ty1 - ty0) * gx" in body  # U's flags
    assert "rows_mass_bits<T, 4>" in body and "rows_mass_bits<T, 8>" in body and "rows_mass_bits<T, 16>" in body
