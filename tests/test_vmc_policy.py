"""Host-side choice between the CG and the sample-space SR solves (CPU)."""

from paper_2204_07816_gb300.vmc import SolverChoice


def test_first_step_and_probes_use_cg():
    c = SolverChoice(n_samples=1024, n_params=4832, probe_every=10)
    assert c.pick(0) == 'cg'
    c.record('cg', 51.1, 556)
    assert c.pick(10) == 'cg' and c.pick(20) == 'cg'


def test_picks_the_cheaper_measured_solver():
    c = SolverChoice(n_samples=1024, n_params=4832)
    c.record('cg', 51.1, 556)          # 0.092 ms per iteration
    c.record('woodbury', 35.7)
    assert c.pick(1) == 'woodbury'
    c.record('cg', 20.5, 205)          # 0.1 ms per iteration, 20.5 ms in all
    assert c.pick(1) == 'cg'


def test_estimate_before_a_measurement_and_size_limit():
    c = SolverChoice(n_samples=4096, n_params=11792, fp64_flops=1e12)
    m = 8192.0
    assert abs(c.woodbury_estimate_ms() - (m * m * 11792 + m ** 3 / 3) / 1e12 * 1e3) < 1e-9
    c.record('cg', 5.6, 12)
    assert c.pick(1) == 'cg'           # 5.6 ms against ~1 s
    big = SolverChoice(n_samples=40000, n_params=100)
    big.record('cg', 1e6, 10000)
    assert big.pick(1) == 'cg'         # beyond the sample-space solve's limit
