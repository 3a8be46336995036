"""The committed ncu summaries are consistent with the bench that reads them:
every summary the bench maps to a kernel and tile exists and names that tile,
and every summary states the command that made it, built from committed
files only."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _kv(path):
    out = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                out[k.strip()] = v.strip()
    return out


def test_bench_profile_table_points_at_matching_summaries():
    import bench
    for (kvar, tile, species, precision), path in bench.PROFILES.items():
        assert os.path.exists(path), path
        kv = _kv(path)
        assert kv["tile"] == f"{tile[0]}x{tile[1]}", path
        assert int(kv["dram_bytes_per_launch"]) > 0
        assert len(kv["kernel_hash"]) == 16
        name = os.path.basename(path)
        assert name.startswith({0: "k_step_register", 2: "k_step_tma", 6: "k_step_smem", 8: "k_step_tile",
                                9: "k_step_bidir", 10: "k_step_ring", 11: "k_step_bidir_jit"}[kvar]), name
        assert ("species" in name) == (species is not None), name
        assert f"_{precision}_" in name, name


def test_every_summary_states_its_command_from_committed_files():
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.txt")):
        text = open(path).read()
        assert re.search(r"command", text), path
        assert "_work" not in text, path
        assert os.path.getsize(path) < 16 * 1024, path
