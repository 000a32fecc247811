"""One filter step and a whole run (oracle; test infrastructure only).

Order within a step (Sec. IV, message schedule, and Sec. II-C):
  (i) prediction and births -> (ii)/(iii) update messages, computed once ->
  beliefs and normalisation -> MMSE estimates and declaration ->
  pruning (the surviving PFs are the legacy set of the next step) ->
  systematic resampling and regularisation of every belief.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import beliefs, messages_dense, messages_woodbury, model, resample


@dataclasses.dataclass
class StepResult:
    pred: model.Predicted
    msg: object
    bel: beliefs.Beliefs
    est: beliefs.Estimate
    keep: np.ndarray
    state: object


def update(pred, params, geom, z, mode: str = "woodbury"):
    if mode == "dense":
        msg = messages_dense.update_messages(pred, params, geom, z)
    else:
        msg = messages_woodbury.update_messages(pred, params, geom, z)
    bel = beliefs.beliefs(pred, msg)
    est = beliefs.estimate(pred, bel, params)
    return msg, bel, est


def step(state, params, geom, z, seed: int, S_max: int, mode: str = "woodbury") -> StepResult:
    pred = model.predict(state, params, geom.J, seed, S_max)
    msg, bel, est = update(pred, params, geom, z, mode)
    keep = beliefs.survivors(est, params) if params.T_pru > 0 else np.arange(pred.S)
    new_state, *_ = resample.resample_and_regularize(pred, bel, keep, params, seed)
    return StepResult(pred=pred, msg=msg, bel=bel, est=est, keep=keep, state=new_state)
