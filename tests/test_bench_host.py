"""Host-side logic of bench.py, without a GPU: the L2 note of the bench line's config,
and the committed steady-state traffic counters the roofline reports."""
import glob
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_l2_note_names_the_buffers_of_the_lattice_timed():
    b = load_bench()
    assert b.l2_note(2048, "f32") == "inputs larger than L2: 2 x 151.0 MB F32 population buffers + 16.8 MB phi plane"
    assert b.l2_note(4096, "bf16dev").startswith("inputs larger than L2: 2 x 302.0 MB 16-bit deviation buffers")
    assert b.l2_note(1024, "f32").startswith("state fits in L2 (79.7 MB")
    assert "but one population buffer smaller" in b.l2_note(2048, "f16dev")
    assert b.l2_note(2048, "f64").startswith("inputs larger than L2: 2 x 302.0 MB F64")


def test_committed_traffic_counters_belong_to_the_current_kernels():
    """Each steady-state traffic file under profiles/ was taken with the step kernels'
    present source (else the bench reports no traffic and the counters must be taken
    again), and its bytes add up."""
    b = load_bench()
    h = b.kernel_source_hash()
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.json")))
    assert files
    for f in files:
        d = json.load(open(f))
        assert d["kernel_source_sha256_16"] == h, f"{os.path.basename(f)}: counters of an older kernel source"
        assert d["dram_bytes_per_launch"] == d["dram_bytes_read_per_launch"] + d["dram_bytes_write_per_launch"]
        assert d["command"].startswith("ncu ") and "--clock-control none" in d["command"]
    q = json.load(open(os.path.join(ROOT, "profiles", "ace_step_quad_f32_2048.json")))
    assert b.stored_traffic("ace_step_quad", "f32", 2048) == q["dram_bytes_per_launch"]
    assert b.stored_traffic("ace_step_quad", "f32", 777) is None
