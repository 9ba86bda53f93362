"""Host logic of bench.py that needs no GPU: the workload descriptions and
the size rules of the batched workload."""
import bench


def test_channel_workload_sizes():
    w = bench.workload()
    assert w["m"] == 3 * 128 * 96 * 128 == 4_718_592
    assert w["n"] == 1000 and w["k"] == 50 and w["l"] == 60 and w["chunk"] == 32
    assert w["bytes_per_step"] == 4 * w["m"] * w["n"]


def test_batched_workload_follows_its_rules():
    ps = bench.batched_problems()
    assert len(ps) == 64
    assert [p["seed"] for p in ps] == list(range(1, 65))
    for b, p in enumerate(ps):
        nx, ny, nz = p["grid"]
        assert nx == nz == 2 * ny                         # m = 3 * 2ny * ny * 2ny
        m = 3 * nx * ny * nz
        assert 40_000 <= m <= 2_100_000                   # U[50k, 2M] rounded to the grid
        assert 64 <= p["n"] <= 512
        assert 10 <= p["k"] <= 80 and p["l"] == p["k"] + 10 <= 90
        assert p["prec"] == ("bf16" if b % 2 else "exact")
    # the same sizes on every call (seeded)
    assert bench.batched_problems() == ps
