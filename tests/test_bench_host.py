"""Host checks of the benchmark's reporting arithmetic (no GPU): the step
roofline rule, the traffic record lookup keyed by the CUDA sources' digest,
and the host description of the CPU baselines."""
import os
import types

import pytest

import bench


def test_roofline_step_is_the_larger_of_atomics_and_bytes():
    ms = types.SimpleNamespace(nx=256, ny=256, nz=64)
    V = ms.nx * ms.ny * ms.nz
    # 5.6 M atomics at 200 G/s = 28 us; bytes 12 * 131072 + 12 * V + 17 * 65536 at 6753 GB/s
    r = bench.roofline_step(5.6e6, 200e9, V, ms, 131072, 6753.0, 80e-6)
    hbm_bytes = 12 * 131072 + 12 * V + 17 * 65536
    assert r["atomic_us"] == pytest.approx(28.0)
    assert r["hbm_us"] == pytest.approx(1e6 * hbm_bytes / 6753e9)
    assert r["roofline_us"] == pytest.approx(max(r["atomic_us"], r["hbm_us"]))
    assert r["serial_roofline_us"] == pytest.approx(r["atomic_us"] + r["hbm_us"])
    assert r["frac"] == pytest.approx(r["roofline_us"] / 80.0)
    # an HBM-bound case: few atomics
    r2 = bench.roofline_step(1e3, 200e9, V, ms, 131072, 6753.0, 80e-6)
    assert r2["roofline_us"] == pytest.approx(r2["hbm_us"])


def test_traffic_record_matches_the_current_sources():
    # the committed record names the digest of the CUDA sources; a lookup
    # for a workload it does not hold gives nothing
    v = bench.profile_traffic("k_ingest", "plain_sequence")
    assert v is None or v > 1e6
    assert bench.profile_traffic("k_ingest", "no_such_workload") is None


def test_traffic_record_ignores_a_stale_digest(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text("kernel=k_ingest workload=w src=0000000000000000 dram_bytes_per_launch=5\n")
    csrc = tmp_path / "paper_2109_13176_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("// kernel\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("k_ingest", "w") is None
    import hashlib
    digest = hashlib.sha256(b"// kernel\n").hexdigest()[:16]
    (prof / "traffic.txt").write_text(f"kernel=k_ingest workload=w src={digest} dram_bytes_per_launch=5\n")
    assert bench.profile_traffic("k_ingest", "w") == 5.0


def test_host_cpu_description():
    h = bench.host_cpu()
    assert h["nproc"] == (os.cpu_count() or 0) and isinstance(h["model"], str) and h["model"]


def test_bench_functions_name_only_defined_globals():
    # every name a function of bench.py loads is a local, a module-level name
    # or a builtin (a missing import would otherwise surface only in a leg
    # that runs on a GPU)
    import ast
    import builtins
    import os
    src = open(os.path.join(os.path.dirname(__file__), "..", "bench.py")).read()
    tree = ast.parse(src)
    top = set()
    for n in tree.body:
        if isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            top.add(n.name)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            top.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, ast.Assign):
            top.update(t.id for t in n.targets if isinstance(t, ast.Name))
    missing = []
    for f in (n for n in tree.body if isinstance(n, ast.FunctionDef)):
        local = set()
        for node in ast.walk(f):
            if isinstance(node, ast.Name) and isinstance(node.ctx, (ast.Store, ast.Del)):
                local.add(node.id)
            elif isinstance(node, (ast.FunctionDef, ast.Lambda)):
                if isinstance(node, ast.FunctionDef):
                    local.add(node.name)
                a = node.args
                local.update(x.arg for x in a.args + a.kwonlyargs + a.posonlyargs)
                local.update(x.arg for x in (a.vararg, a.kwarg) if x)
            elif isinstance(node, (ast.Import, ast.ImportFrom)):
                local.update((a.asname or a.name).split(".")[0] for a in node.names)
            elif isinstance(node, ast.ExceptHandler) and node.name:
                local.add(node.name)
        for node in ast.walk(f):
            if isinstance(node, ast.Name) and isinstance(node.ctx, ast.Load):
                if node.id not in local and node.id not in top and not hasattr(builtins, node.id):
                    missing.append((f.name, node.id, node.lineno))
    assert not missing, missing


def test_traffic_digest_follows_the_kernels_own_sources(tmp_path, monkeypatch):
    # a kernel's DRAM bytes stay valid while its own .cu file and the headers
    # are unchanged; another kernel's file does not matter
    csrc = tmp_path / "paper_2109_13176_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "ingest.cu").write_text("// walk\n")
    (csrc / "extract.cu").write_text("// columns\n")
    (csrc / "gvom_internal.h").write_text("// shared\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.source_digest("k_march")
    (csrc / "extract.cu").write_text("// columns, changed\n")
    assert bench.source_digest("k_march") == d0
    assert bench.source_digest("k_columns_tma") != d0
    (csrc / "ingest.cu").write_text("// walk, changed\n")
    assert bench.source_digest("k_march") != d0
    d1 = bench.source_digest("k_march")
    (csrc / "gvom_internal.h").write_text("// shared, changed\n")
    assert bench.source_digest("k_march") != d1
