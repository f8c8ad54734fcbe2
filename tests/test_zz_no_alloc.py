"""The allocation-free transform entry point against the scene build's own transform.

ags_transform_vertices_noalloc serves callers that cannot let the library call
cudaMalloc (device memory reserved up front by their own allocator, or no
room for the synchronisation an allocation may cause mid-work). It keeps its
scratch in a fixed device array inside the library. This file is collected
last so that a failure here never hides the other GPU tests.
"""
import numpy as np
import pytest
import torch

import paper_2503_01471_gb300 as ags
from paper_2503_01471_gb300 import build as B
from paper_2503_01471_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = ags.ags_context_create(0)
    yield c
    ags.ags_context_destroy(c)


def _scene(seed):
    rng = np.random.default_rng(seed)
    envs = []
    for e in range(3):
        objs = []
        for k in range(int(rng.integers(5, 25))):
            v = rng.uniform(-3, 3, (int(rng.integers(3, 40)), 3)).astype(np.float32)
            f = rng.integers(0, v.shape[0], (int(rng.integers(1, 20)), 3)).astype(np.int32)
            q = rng.normal(size=4) * rng.uniform(0.3, 2.0)
            p = rng.uniform(-15, 15, 3)
            objs.append((v, f, np.concatenate([p, q]).astype(np.float32), k))
        envs.append(objs)
    return S.scene_from_lists(envs)


def _via_build(ctx, batch):
    """World triangles [F,9] of every env, from the existing entry points."""
    scene = ags.ags_scene_build(ctx, batch)
    try:
        return np.concatenate([ags.ags_scene_get_world_triangles(scene, e)[0] for e in range(batch.n_envs)])
    finally:
        ags.ags_scene_destroy(scene)


def _via_noalloc(ctx, batch, out):
    base = torch.as_tensor(batch.vertices).cuda()
    offs = torch.as_tensor(batch.sub_vert.astype(np.int32)).cuda()
    poses = torch.as_tensor(batch.poses).cuda()
    ags.ags_transform_vertices_noalloc(ctx, base, offs, poses, out)
    torch.cuda.synchronize()
    w = out[: base.shape[0], :3].cpu().numpy()
    # global vertex index of every triangle corner (indices are local to their sub-mesh)
    sub_of_tri = np.repeat(np.arange(batch.sub_seg.shape[0]), np.diff(batch.sub_tri))
    gidx = batch.indices.astype(np.int64) + batch.sub_vert[sub_of_tri][:, None]
    return w[gidx].reshape(-1, 9)


def _via_oracle(batch):
    """FP64 world triangles [F,9] of every env from the oracle's own transform."""
    import oracle as O
    out = []
    for e in range(batch.n_envs):
        vs, ix, ps, sg = batch.env_submeshes(e)
        out.append(O.world_triangles(vs, ix, ps, sg)[0])
    return np.concatenate(out)


def test_noalloc_transform_matches_build_on_two_calls(ctx):
    a, b = _scene(1), _scene(2)
    vmax = max(a.vertices.shape[0], b.vertices.shape[0])
    out = torch.full((vmax, 4), float("nan"), device="cuda")
    for batch in (a, b):  # two calls in a row share the scratch array
        ref = _via_build(ctx, batch)
        got = _via_noalloc(ctx, batch, out)
        assert np.array_equal(got, ref)  # the existing entry point's kernels: identical
        # and within 1 ulp of the FP64 transform of the oracle (the transform tests' bound)
        exact = _via_oracle(batch)
        ulp = np.spacing(np.maximum(np.abs(exact), 1.0).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got.astype(np.float64) - exact) <= ulp)


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    base = torch.zeros((4, 3), device="cuda")
    offs = torch.zeros(65538, dtype=torch.int32, device="cuda")
    offs[-1] = 4
    poses = torch.zeros((65537, 7), device="cuda")
    poses[:, 6] = 1.0
    out = torch.zeros((4, 4), device="cuda")
    with pytest.raises(ags.AgsError, match="65536"):
        ags.ags_transform_vertices_noalloc(ctx, base, offs, poses, out)


def test_noalloc_checks_shapes_and_dtypes_on_the_host(ctx):
    base = torch.zeros((8, 3), device="cuda")
    offs = torch.tensor([0, 4, 8], dtype=torch.int32, device="cuda")
    poses = torch.zeros((2, 7), device="cuda")
    poses[:, 6] = 1.0
    out = torch.zeros((8, 4), device="cuda")
    bad = [
        dict(submesh_vertex_offsets=offs[:2]),                     # J entries instead of J+1
        dict(submesh_vertex_offsets=offs.to(torch.int64)),         # wrong dtype
        dict(world_vertices=out[:7]),                              # fewer rows than vertices
        dict(world_vertices=torch.zeros((8, 3), device="cuda")),   # not [V,4]
        dict(poses=torch.zeros((2, 6), device="cuda")),            # not [J,7]
        dict(base_vertices=base.double()),                         # wrong dtype
        dict(base_vertices=base.cpu()),                            # host tensor
    ]
    for kw in bad:
        args = dict(base_vertices=base, submesh_vertex_offsets=offs, poses=poses, world_vertices=out)
        args.update(kw)
        with pytest.raises(ValueError):
            ags.ags_transform_vertices_noalloc(ctx, **args)
    ags.ags_transform_vertices_noalloc(ctx, base, offs, poses, out)  # the well-formed call still runs
    torch.cuda.synchronize()
    assert torch.equal(out[:, :3], base)
