"""The bench's JSON line on the CPU: the reference arm (the oracle, timed on the host cores) on a small droplet,
alone and under a two-process launch (rank 0 prints the one line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def check_line(d, n_gpus, n=32):
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["n_gpus"] == n_gpus
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "Mpts/s" and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert "workload" in d["config"] and d["config"]["grid"] == [n, n, n]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "32", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    check_line(json.loads(lines[0]), 1)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_two_ranks():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]  # (the launcher would take a script's --n for one of its own options)
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    check_line(json.loads(lines[0]), 2, n=128)


def test_bench_manufactured_stencil_is_the_mac_operator():
    """The plain-PyTorch stencil the bench uses to manufacture f = L p* for its error statements equals the
    oracle's MAC operator (periodic x, y; Neumann z; stretched z)."""
    torch = pytest.importorskip("torch")
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1907_00890_gb300 import synth
    n = (12, 10, 9)
    dz = synth.stretched_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 0.8 / n[1], dz, ("P", "P", "NN"))
    p = synth.rng(5).standard_normal(g.shape)
    got = bench._torch_laplacian_ppnn(torch, torch.tensor(p), 1.0 / n[0], 0.8 / n[1], dz).numpy()
    want = oracle.apply_laplacian(g, p)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_record_traffic_from_an_ncu_launch_list(tmp_path):
    """bench.py --record-traffic turns an ncu launch list (CSV, base units) into DRAM bytes per launch and
    kernel class, keyed to the current sources, instead of numbers typed in by hand."""
    sys.path.insert(0, ROOT)
    import bench
    hdr = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
          '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"'
    rows = []
    launches = [(0, "k_xinv<double, double2>(vofp::XInvArgs)", 60000, 1.0e7, 7.0e6),
                (1, "k_xinv<double, double2>(vofp::XInvArgs)", 62000, 1.1e7, 7.0e6),
                (2, "k_ypass_tma<float, true, 8, 4>(vofp::YTmaArgs, CUtensorMap_st)", 30000, 4.0e6, 4.0e6),
                (3, "k_xfwd<double, double2, 1>(vofp::XArgs)", 90000, 5.0e7, 1.7e7)]
    for i, name, ns, rd, wr in launches:
        for m, u, v in (("dram__bytes_read.sum", "byte", rd), ("dram__bytes_write.sum", "byte", wr),
                        ("gpu__time_duration.sum", "nsecond", ns)):
            rows.append('"%d","1","python","h","%s","1","7","(256, 1, 1)","(64, 1, 1)","0","10.3","","%s","%s","%s"'
                        % (i, name, m, u, "{:,}".format(int(v))))
    csv_path = tmp_path / "launches.csv"
    csv_path.write_text("==PROF== Connected\n" + hdr + "\n" + "\n".join(rows) + "\n")
    out = tmp_path / "traffic.json"

    class A:
        record_traffic = str(csv_path)
        traffic_workload = "w"
        traffic_out = str(out)
    bench.record_traffic(A)
    t = json.loads(out.read_text())
    assert t["source_sha"] == bench.source_sha()
    assert t["workloads"]["w"] == {"x_inverse": 17500000, "y_inverse": 8000000, "x_forward_div": 67000000}
