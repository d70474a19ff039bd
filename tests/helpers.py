"""Shared test helpers: parity metrics and the GPU-availability gate."""
import numpy as np

# per-moment floors of the error normalisation: O(1) quantities use their own
# max, small ones (velocities, shear stress, heat flux) at least 1e-2
FLOORS = np.array([1.0, 1e-2, 1e-2, 1.0, 1.0, 1.0, 1.0, 1e-2, 1e-2, 1e-2])


def moment_errors(m: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """e_k = max_s |m_k - ref_k| / max(max_s |ref_k|, floor_k), k over the 10 moments."""
    scale = np.maximum(np.max(np.abs(ref), axis=1), FLOORS)
    return np.max(np.abs(m - ref), axis=1) / scale


def weighted_state_error(f: np.ndarray, ref: np.ndarray, w: np.ndarray) -> float:
    """max |w (f - ref)| / max |w ref| over fields, velocities and nodes."""
    ww = w[None, :, None]
    return float(np.max(np.abs(ww * (f - ref))) / np.max(np.abs(ww * ref)))


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False
