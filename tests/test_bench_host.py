"""Host logic of bench.py that needs no GPU: the JSON line of the reference arm
(the CPU oracle, run as the driver runs it, on a small lattice) and the rule
that reports the recorded DRAM traffic only for the kernel, tile and workload
it was measured on."""

import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--dims", "8,8,8,8", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "GFlop/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["scaling"] == "weak" and d["data"] == "synthetic" and d["dtype"] == "f64"
    assert d["config"]["workload"] == "mobius_dwf_dhop_8x8x8x8_ls12_f32"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "4096 random 4D sites" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GFlop/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def _record(path, tile="2,128,7,4,6", dims="32,32,32,64", Ls=12, digest=None):
    with open(path, "w") as f:
        f.write("# record\n\n- tile: %s\n- dims: %s\n- Ls: %d\n- source_digest: %s\n"
                "- dram_read_bytes: 4.5e9\n- dram_write_bytes: 2.4e9\n"
                % (tile, dims, Ls, digest or bench.kernel_digest()))


def test_recorded_traffic_only_for_its_kernel_tile_and_workload(tmp_path, monkeypatch):
    rec = tmp_path / "record.md"
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    tile, dims = (2, 128, 7, 4, 6), (32, 32, 32, 64)
    assert bench.recorded_traffic(tile, dims, 12) is None  # no record
    _record(rec)
    assert bench.recorded_traffic(tile, dims, 12) == 6.9e9
    assert bench.recorded_traffic((2, 128, 6, 4, 6), dims, 12) is None  # other tile
    assert bench.recorded_traffic(tile, (32, 32, 16, 32), 12) is None  # other lattice
    assert bench.recorded_traffic(tile, dims, 16) is None  # other Ls
    _record(rec, digest="0" * 16)  # the stencil sources changed since the capture
    assert bench.recorded_traffic(tile, dims, 12) is None


def test_algorithmic_bytes_per_site_update():
    # FP32: 4 * (48 + 72 / (Ls nrhs)) -- 216 B at Ls = 12, 194 B for 12 RHS
    assert bench.bytes_per_site(4, 12) == 216.0
    assert bench.bytes_per_site(4, 12, 12) == 4 * (48 + 0.5)
    assert bench.bytes_per_site(8, 16) == 420.0


def test_profiling_options_need_main_only():
    # --op, --prec and --nrhs select what a profiling run (--main-only) times;
    # the default benchmark line refuses them before touching the GPU
    import subprocess
    import sys
    for extra in (["--op", "d"], ["--prec", "f16"], ["--nrhs", "2"]):
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + extra,
                           capture_output=True, text=True, timeout=120)
        assert r.returncode == 2 and "--main-only" in r.stderr, (extra, r.stderr[-300:])


def test_kernel_digest_follows_code_not_comments(tmp_path, monkeypatch):
    # the traffic record is voided by a change of the stencil code, not by an
    # edited comment or reflowed whitespace
    csrc = tmp_path / "paper_2112_01852_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (csrc / "dw_common.cuh").write_text("// common\nstruct A { int x; };\n")
    (csrc / "dw_dslash.cuh").write_text("/* kernel */\nint f(int a) { return a + 1; }\n")
    (csrc / "dw_api.cu").write_text("int host_side() { return 0; }\n")
    d0 = bench.kernel_digest()
    (csrc / "dw_dslash.cuh").write_text("/* the kernel, reworded */\nint f(int a)\n"
                                        "{  return a + 1;  // same code\n}\n")
    (csrc / "dw_api.cu").write_text("int host_side() { return 1; }\n")  # not a stencil file
    assert bench.kernel_digest() == d0
    (csrc / "dw_dslash.cuh").write_text("int f(int a) { return a + 2; }\n")
    assert bench.kernel_digest() != d0
