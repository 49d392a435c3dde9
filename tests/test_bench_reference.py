"""bench.py's reference arm (the oracle timed on the host cores) on CPU: one
JSON line with the contract's keys, on the same workload config as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--classes", "1,1,1,1", "2,1,0,3", "--cpu-seconds", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Gints/s" and d["higher_is_better"]
    assert set(d["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    sys.path.insert(0, ROOT)
    import bench

    class A:
        npair, naux = 4096, 512
    assert d["config"] == bench.sweep_config(A, [(1, 1, 1, 1), (2, 1, 0, 3)], 1)


def test_gpu_arm_line_stays_small():
    """The GPU arm's JSON line for the full 525-class sweep with every
    one-off field stays under 4 KB (a driver keeps the tail of long lines)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2210_03192_gb300 import workloads as W

    class A:
        npair, naux, steps, warmup, hints, hrr_hints = 4096, 512, 20, 5, 103, 120
    classes = list(W.SWEEP_CLASSES)
    table = [dict(cls=c, ms=123.4567, gints_s=12.3456, gflops=789.12, frac=0.61234) for c in classes]
    clk = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 1234}
    xclk = [2070.0, 1234, []]
    res = dict(ms=1234567.8, total_int=192675840000 * 20, total_flops=1e15, table=table, clocks=clk,
               launches=38220, roofline=dict(bound="alu", achieved=921.46, peak=1258.6, unit="GFLOP/s", frac=0.7322,
                                             traffic=17140105216, kernel="eri3c_kernel, class (44|6) K_ab=6",
                                             peak_source="derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                                             flops_per_launch=1707283054592.0, launch_ms=1852.808),
               l3_frac=dict(classes=495, min=0.3585, median=0.5872, at_least_half=411),
               e2e=dict(value=2.2189, unit="Gints/s", h2d_bytes_per_step=398458880,
                        d2h_bytes_per_step=1541406720000, seconds=86.834,
                        host_buffer="huge-page mapping, cudaHostRegister"))
    cpu = dict(value=0.013287, unit="Gints/s", cores=16, kind="oracle",
               sample="3 pairs x 64 ket shells of each of 525 classes (17640000 integrals), McMurchie-Davidson "
                      "FP64, 13.3 s")
    extras = dict(
        fp64_peak_measured=dict(gflops=1190.2, ms=150.1, frac_of_derived=0.9457, method="lx3c_fp64_rate",
                                clocks=xclk),
        config1=dict(workload="(pp|d) 64x32", integrals=92160, ms=0.0637, gints_s=1.4473,
                     frac=0.0176, launches=4, reps=20000, clocks=xclk),
        dfj=dict(workload="DF-J 256 atoms", nao=7680, naux_ao=27136,
                 screened_triples=14074753270, integrals=324312871258.0, tile_fill=0.9728, setup_s=8.81,
                 fused_s=54.314, gamma_only_s=53.001, J_only_s=53.24, fused_frac=0.4987,
                 launches=217,
                 contracted=dict(setup_s=9.12, fused_s=41.234, gamma_only_s=40.123, J_only_s=40.456,
                                 flops_ratio=0.7123, fused_frac=0.4567, speedup=1.317, launches=870),
                 clocks=xclk),
        batch=dict(workload="16 molecules, 20-400 atoms",
                   screened_triples=5238364893.0, plan_s=4.99, bind_capture_s=0.61, graph_branches_s=32.432,
                   per_class_s=32.661, graph_persistent_s=58.32,
                   frac=dict(graph_branches=0.4941, per_class=0.4907, graph_persistent=0.2748),
                   launches=dict(per_class=6127, graph_branches_kernel_nodes=6127, graph_persistent_kernel_nodes=3377,
                                 persistent_tiers=2),
                   speedup_graph_vs_per_class=1.007, clocks=xclk),
        grad=dict(workload="dE/dR, 64 atoms", screened_triples=206219480,
                  fwd_ms=1276.6, bwd_ms=5431.13, fwd_bwd_ms=6707.3, plain_fwd_gamma_J_ms=1325.64,
                  fwd_bwd_over_fwd=5.254, bwd_frac=0.5027, launches=dict(fwd=331, bwd=984), clocks=xclk),
        metric=dict(workload="metric, 256-atom aux basis", naux_ao=27136,
                    metric_ms=37.88, metric_frac=0.4952, cholesky_ms=6106.63, cholesky_gflops=1090.7,
                    cholesky_frac=0.8666, cholesky_dropped=1234, solve_ms=138.62,
                    metric_launches=48, clocks=xclk),
        dfj_multi=dict(workload="DF-J 32 atoms", screened_triples=123456789,
                       nd1_ms=1234.5, nd8_ms=2345.6, per_density_ms_nd8=293.2, per_density_speedup=4.21,
                       nd1_contracted_ms=987.65, clocks=xclk))
    line = bench.make_line(A, res, classes, 1, cpu, extras)
    text = json.dumps(line, separators=(",", ":"))
    assert len(text) < 3800, len(text)  # margin below 4 KB
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "clocks", "gpu_launches", "e2e"):
        assert k in line, k
