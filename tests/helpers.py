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


def particle_errors(xu_g, xu_r, v_g, v_r, x0):
    """Largest per-particle relative errors, element by element: position
    error over the particle's own displacement |X_ref - X_0|, velocity error
    over its own speed |V_ref| (3-vector norms), each denominator floored at
    its rms over the particles compared.  The floors: a position error is
    the sum of the per-step errors of the displacement increments, so it
    scales with the distance travelled, and two correct FP64 trajectories
    already differ by the rounding of the position itself (up to ulp(L)/2 per
    step), which a particle that ended near its start would divide by ~0; a
    velocity error scales with the fluid speed at the particle (field and
    interpolation rounding), not with the particle's own speed.  Against the
    norm-wise errors this is the max norm: one particle off by ten times the
    bar fails it whatever the others do."""
    d = np.linalg.norm(xu_r - x0, axis=0)
    s = np.linalg.norm(v_r, axis=0)
    fd = np.sqrt(np.mean(d ** 2)) if d.size else 1.0
    fs = np.sqrt(np.mean(s ** 2)) if s.size else 1.0
    px = np.linalg.norm(xu_g - xu_r, axis=0) / np.maximum(d, max(fd, 1e-300))
    pv = np.linalg.norm(v_g - v_r, axis=0) / np.maximum(s, max(fs, 1e-300))
    return (float(px.max()) if px.size else 0.0), (float(pv.max()) if pv.size else 0.0)


def traj_errors(x_gpu, img_gpu, v_gpu, ids_gpu, ref: oracle.State, x0):
    """Relative errors of unwrapped positions (relative to the displacement)
    and velocities, in id order: (e_x, e_v) norm-wise over all particles and
    (p_x, p_v) the largest per-particle errors (particle_errors).  Every
    trajectory test bounds all four by its bar."""
    xg, vg, ig = by_id(ids_gpu, x_gpu, v_gpu, img_gpu)
    xr, vr, ir = by_id(ref.ids, ref.x, ref.v, ref.img)
    xu_g = xg + L * ig
    xu_r = xr + L * ir
    ex = np.linalg.norm(xu_g - xu_r) / np.linalg.norm(xu_r - x0)
    ev = np.linalg.norm(vg - vr) / np.linalg.norm(vr)
    px, pv = particle_errors(xu_g, xu_r, vg, vr, x0)
    print(f"trajectory errors: e_x {ex:.3e} e_v {ev:.3e}, per particle {px:.3e} {pv:.3e}")
    return ex, ev, px, pv


def assert_same_storage(st, ref: oracle.State, N, P, brick=1):
    """Per-subdomain id lists equal; where they differ, every differing
    particle must sit within rounding of a cell face on one side (its key
    depends on the ulp-level trajectory difference).  Returns the number of
    storage slots that differ (0 when the lists are equal)."""
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
    # a particle straddles a face only when it lies within ~1e-13 of it: the
    # expected count is far below one, so more than a few is a fault
    assert len(bad) <= max(4, ids.size // 10000), f"{len(bad)} storage slots differ"
    print(f"storage slots differing at cell faces: {len(bad)} of {ids.size}")
    return len(bad)
