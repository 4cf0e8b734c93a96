"""The benchmark's algorithmic units (no GPU): per env-step of the 17x17x9
block (V 2601, E 13864, T 10240; 10 substeps x 1 iteration) the shared-memory
bytes, FP32 operations and HBM bytes that the roofline divides by are the
stated per-constraint and per-vertex figures, and they scale with substeps,
iterations and mesh size as the definitions say."""
import bench
from paper_2503_18616_gb300 import inputs

V, E, T = 2601, 13864, 10240


def test_shared_memory_bytes_per_env_step():
    p = inputs.default_params()
    got = bench.smem_bytes_per_env_step(V, E, T, p)
    # float4 load + store of both edge ends, all four tet corners, and one
    # load + store per vertex in the fused collision / prediction pass
    assert got == 10 * (E * 2 * 2 * 16 + T * 2 * 4 * 16 + V * 2 * 16)
    assert abs(got / 1e6 - 22.8) < 0.05
    p2 = inputs.default_params(iterations=3, substeps=5)
    assert bench.smem_bytes_per_env_step(V, E, T, p2) == 5 * (3 * (E * 64 + T * 128) + V * 32)


def test_fp32_operations_and_hbm_bytes_per_env_step():
    p = inputs.default_params()
    assert abs(bench.flops_per_env_step(V, E, T, p) / 1e6 - 16.9) < 0.1
    assert bench.BYTES_VERT == 48     # x and v, read and written once per step, float32 x 3
    assert bench.BYTES_VERT * V == 124848


def test_units_scale_linearly_with_the_mesh():
    p = inputs.default_params()
    a = bench.smem_bytes_per_env_step(V, E, T, p)
    b = bench.smem_bytes_per_env_step(2 * V, 2 * E, 2 * T, p)
    assert b == 2 * a
    fa = bench.flops_per_env_step(V, E, T, p)
    assert bench.flops_per_env_step(2 * V, 2 * E, 2 * T, p) == 2 * fa


def test_every_workload_builds_its_batch_and_oracle_meshes():
    """Every named workload yields meshes, parameters and oracle meshes (with
    the connection radius the workload sets), without a GPU."""
    for name in inputs.WORKLOADS:
        b = bench.Batch(name, n_env_override=8)
        assert b.n_env == 8 and len(b.meshes) >= 1
        assert b.describe()
        om = b.oracle_mesh(b.mesh_index(0))
        assert om.V == b.verts(0)
        if b.params.get("conn_radius", 0.0) > 0:
            assert om.C > 0 and b.params["tool_model"] == 1


def test_algorithmic_shared_memory_bytes_follow_the_method():
    """The roofline's numerator: per projection the 12-byte positions of the
    touched vertices read and written (48 B per edge, 96 B per tet), so the
    4096-env launch of the 17x17x9 block moves 67.5 GB; the kernel's float4
    traffic (w in the fourth lane) is reported beside it, not instead."""
    p = inputs.default_params()
    per = bench.smem_alg_bytes_per_env_step(V, E, T, p)
    assert per == 10 * (E * 48 + T * 96)
    assert abs(per * 4096 / 1e9 - 67.52) < 0.01
    assert bench.smem_alg_bytes_per_env_step(V, E, T, dict(p, iterations=3)) == 3 * per
    pg = inputs.default_params(tool_model=1)
    assert bench.smem_alg_bytes_per_env_step(V, E, T, pg, C=7, F=11) == 10 * (E * 48 + T * 96 + 7 * 96 + 11 * 36)
    assert bench.NET_FLOP_ROW == 10496   # 2 x (960 + 4096 + 192)
