"""Shared helpers of the parity tests: run the CUDA path and the oracle on the
same seeded inputs and compare them."""
import numpy as np

import oracle
import synth

L = synth.L_BOX


def by_id(ids, *arrays):
    """Reorder (3, n) / (n,) arrays from storage order to particle-id order."""
    order = np.argsort(np.asarray(ids, dtype=np.int64), kind="stable")
    return [a[..., order] for a in arrays]


def gpu_state(sim, ens=0):
    st = sim.get_state(ens=ens, device="cpu")
    return {k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in st.items()}


def traj_errors(x_gpu, img_gpu, v_gpu, ids_gpu, ref: oracle.State, x0):
    """Norm-wise relative errors of unwrapped positions (relative to the
    displacement) and velocities, in id order."""
    xg, vg, ig = by_id(ids_gpu, x_gpu, v_gpu, img_gpu)
    xr, vr, ir = by_id(ref.ids, ref.x, ref.v, ref.img)
    xu_g = xg + L * ig
    xu_r = xr + L * ir
    ex = np.linalg.norm(xu_g - xu_r) / np.linalg.norm(xu_r - x0)
    ev = np.linalg.norm(vg - vr) / np.linalg.norm(vr)
    return ex, ev, np.abs(xu_g - xu_r).max(), np.abs(vg - vr).max()


def assert_same_storage(st, ref: oracle.State, N, P, brick=1):
    """Per-subdomain id lists equal; where they differ, every differing
    particle must sit within rounding of a cell face on one side (its key
    depends on the ulp-level trajectory difference)."""
    assert np.array_equal(st["seg"], ref.seg), (st["seg"], ref.seg)
    ids = st["ids"].astype(np.uint32)
    if np.array_equal(ids, ref.ids):
        return 0
    bad = np.nonzero(ids != ref.ids)[0]
    for p in np.concatenate([ids[bad], ref.ids[bad]]):
        xg = st["x"][:, ids == p][:, 0]
        xr = ref.x[:, ref.ids == p][:, 0]
        cg = np.floor(xg * (N / L))
        cr = np.floor(xr * (N / L))
        near = np.abs(xg - xr).max() < 1e-9 and np.any(cg != cr)
        assert near, f"particle {p} placed differently without straddling a face"
    return len(bad)
