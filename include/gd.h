/*
 * gd.h -- C ABI of the B300 batched driving-simulator step.
 *
 * A batch of independent worlds (GPUDrive, arXiv 2408.01584, Sec. 3.1:
 * many worlds with their own agent counts stepped in parallel on one
 * accelerator) is uploaded once by gd_create and then advanced on the GPU:
 *
 *   gd_step     kinematic bicycle dynamics (App. B), agent/agent and
 *               agent/road-edge collision (Sec. 3.1, Sec. 3.2 "Termination
 *               conditions"), goal reward (Sec. 3.2 "Rewards"), done flags
 *               and the end of each world's episode; worlds whose episode
 *               ended are reset first when GD_AUTO_RESET is set;
 *   gd_observe  each agent's ego-frame observation: the K nearest road
 *               points and P nearest other agents within the observation
 *               radius (Sec. 3.2 "Sensor modalities"; 50 m in Fig. 1);
 *   gd_step_observe, gd_rollout   the same in one call, and whole episodes;
 *   gd_observe_lidar, gd_step_observe_lidar, gd_rollout_lidar   the LiDAR
 *               and view-cone observations (Sec. 3.2 "Sensor modalities":
 *               rays cast against bounding boxes and road edges, all around
 *               or in a cone turned by a head-rotation action);
 *   gd_invert_actions   expert actions that reproduce a trajectory (Sec. 3.2
 *               "Agent dynamics": exact under the simplified invertible
 *               model, heading and speed under the kinematic bicycle);
 *   gd_rollout_backward / gd_step_backward   adjoint of the dynamics, the
 *               ego-frame observation and a smooth goal-distance reward (the
 *               paper has no gradient; this is an extension).
 *
 * Conventions
 *   - Units are SI (m, s, rad).  Agents and road points are given in
 *     compressed-sparse-row order: world w owns agents agent_off[w] ..
 *     agent_off[w+1]-1 and road points road_off[w] .. road_off[w+1]-1.
 *     "Local" indices count from the start of the world's range.
 *   - Every per-step pointer argument is DEVICE memory owned by the caller,
 *     contiguous, 16-byte aligned for float arrays of 4 or more columns.
 *     Scene arrays passed to gd_create are HOST memory and are copied.
 *   - All calls are asynchronous on the stream given to gd_create except
 *     gd_sync, gd_destroy and gd_create itself; none of them synchronises
 *     the device unless stated.
 *   - Errors are status codes, never exceptions.  Arguments are validated
 *     before anything is launched; a call that returns an error has
 *     launched nothing.  gd_last_error(env) returns a message for the last
 *     error of that env (gd_last_error(NULL): the last gd_create error of
 *     the calling thread).  Faults found on the device (a non-finite
 *     action, a steering angle with |delta| >= pi/2 under the kinematic
 *     bicycle) set a sticky error word that gd_sync reports.
 *   - Observation row layout (float32, F = 8 + 8P + 4K columns):
 *       ego[8]       = (v, length, width, goal_x', goal_y', collided,
 *                       offroad, goal_reached)
 *       partner[P][8]= (x', y', cos(dtheta), sin(dtheta), v, length,
 *                       width, 1)
 *       road[K][4]   = (x', y', road type, 1)
 *     where (x', y') is the offset from the agent rotated by -theta.
 *     Slots are sorted by (squared distance, local index); unused slots are
 *     all zero.  The row of a done agent is all zero except the three flags.
 */
#ifndef GD_H
#define GD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gd_status {
  GD_OK = 0,
  GD_ERR_INVALID_ARG = 1,  /* bad argument, bad scene, or a device-detected bad action */
  GD_ERR_CUDA = 2,         /* a CUDA runtime call failed (message has the CUDA error) */
  GD_ERR_OOM = 3,          /* device or host allocation failed */
  GD_ERR_CAPACITY = 4,     /* a size exceeds a compiled limit (see GD_MAX_*) */
  GD_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  GD_ERR_STATE = 6         /* call not valid in the env's current state */
} gd_status;

/* gd_config.dynamics */
#define GD_DYN_BICYCLE 0      /* kinematic bicycle model, App. B (default); steer = wheel angle (rad) */
#define GD_DYN_INVERTIBLE 1   /* simplified invertible model, Sec. 3.2 "Agent dynamics"; steer = curvature (1/m) */

/* gd_config.flags */
#define GD_TERM_COLLISION 0x1u   /* agent/agent collision ends the agent's episode (Sec. 3.2) */
#define GD_TERM_OFFROAD 0x2u     /* crossing a road edge ends the agent's episode (Sec. 3.2) */
#define GD_AUTO_RESET 0x4u       /* gd_step first resets worlds whose episode ended */
#define GD_BATCHED 0x8u          /* persistent kernels: the step over a world work list, the observation
                                    over an agent counter (or fused with the step, obs_split = 0) */
#define GD_DIFFERENTIABLE 0x10u  /* keep checkpoints for gd_rollout_backward, each agent's K-th road
                                    distance at every step of gd_rollout_objective (4 B x A x
                                    episode_len) and its road selection (2 B x K x A x episode_len,
                                    taken at gd_create when it fits; the backward pass reads it instead
                                    of selecting again, else re-selects within the K-th distance) */
#define GD_NONTRIVIAL_INIT 0x20u /* "all nontrivial" initialisation (Sec. 3.2 "Simulator sharp-edges"):
                                    agents within nontrivial_dist of their goal at the start are not
                                    controlled (GD_FLAG_STATIC); the observation keeps such parked
                                    agents' road selections between steps (4 B x K x A) */

/* per-agent status byte (gd_get_state / gd_set_state) */
#define GD_FLAG_DONE 0x1u
#define GD_FLAG_GOAL 0x2u
#define GD_FLAG_COLLIDED 0x4u
#define GD_FLAG_OFFROAD 0x8u
#define GD_FLAG_STATIC 0x10u   /* not controlled: does not move, is not scored, reports done = 1, and
                                  stays in the scene (an obstacle, a partner, a LiDAR target); a
                                  world's episode ends when its controlled agents are done */

/* road point types and agent types */
#define GD_ROAD_LANE 0
#define GD_ROAD_EDGE 1
#define GD_AGENT_VEHICLE 0
#define GD_AGENT_CYCLIST 1
#define GD_AGENT_PEDESTRIAN 2

/* compiled limits */
#define GD_MAX_AGENTS_PER_WORLD 128
#define GD_MAX_K_ROAD 256
#define GD_MAX_PARTNERS 127
#define GD_MAX_ROAD_PER_WORLD 32767
#define GD_MAX_LIDAR_RAYS 8192

typedef struct gd_config {
  int32_t k_road;            /* K road slots per observation, 0..GD_MAX_K_ROAD */
  int32_t n_partners;        /* P partner slots, 0..GD_MAX_PARTNERS */
  int32_t episode_len;       /* steps per episode (91 at 10 Hz) */
  int32_t ckpt_every;        /* checkpoint interval of differentiable rollouts (10) */
  float obs_radius;          /* m, radius filter (50) */
  float goal_radius;         /* m, goal reached when distance <= this (2) */
  float dt;                  /* s (0.1) */
  float v_max;               /* m/s, speed clip of App. B (30) */
  float collision_penalty;   /* subtracted from the reward on collision (0) */
  float offroad_penalty;     /* subtracted from the reward off road (0) */
  float smooth_c;            /* m, scale of the smooth goal reward (1) */
  uint32_t flags;            /* GD_TERM_* | GD_AUTO_RESET | GD_BATCHED | GD_DIFFERENTIABLE | GD_NONTRIVIAL_INIT */
  int32_t block_size;        /* threads per block of the batched step kernel (and of the fused
                                observation); 0 = default (256), 128, 256 or 512 */
  float road_cell;           /* m, road-point grid cell; 0 = default (8) */
  int32_t topk_strategy;     /* road top-K method: 0 = default, 1 = bucket rank, 2 = bitonic sort */
  int32_t lidar_rays;        /* rays per agent of the LiDAR observation, 0..GD_MAX_LIDAR_RAYS;
                                0 = LiDAR not enabled (default); 3000 in Fig. 1 */
  float lidar_fov;           /* rad, width of the ray fan, in [1e-3, 2 pi]: 2 pi = LiDAR (default),
                                2 pi / 3 = the 120-degree view cone of Fig. 1 */
  int32_t lidar_block_size;  /* threads per block of the fused LiDAR kernel: 0 = default (256),
                                128, 256 or 384 */
  int32_t lidar_no_tile;     /* 1: the fused LiDAR kernel reads the road from global memory
                                instead of a shared-memory tile (more warps per SM); default 0 */
  int32_t lidar_split;       /* 1: with GD_BATCHED the step and the LiDAR scan are two launches
                                (the scan over all agents at once); default 0 = one fused launch */
  int32_t dynamics;          /* GD_DYN_BICYCLE (default) or GD_DYN_INVERTIBLE: the simplified model,
                                a double integrator along the heading of the start of the step,
                                ds = v dt + a dt^2 / 2, x += cos(theta) ds, y += sin(theta) ds,
                                theta += steer * ds, v += a dt (no speed clip; length unused) */
  float nontrivial_dist;     /* m, with GD_NONTRIVIAL_INIT: agents at most this far from their goal
                                at the start are not controlled (2; Sec. 3.2) */
  int32_t road_no_tile;      /* 1: the fused and adjoint kernels read each world's road block from
                                global memory instead of copying it into shared memory (more CTAs per
                                SM); default 0 */
  int32_t obs_split;         /* radial observation with GD_BATCHED: 1 (default) = the step (a
                                persistent kernel over worlds) then the observation (a persistent
                                kernel over agents, no per-world barriers) as two launches; 0 = both
                                in one fused launch.  Both give identical results, objective terms of
                                gd_rollout_objective included. */
  int32_t adjoint_split;     /* adjoint of a step (GD_DIFFERENTIABLE): 1 (default) = two launches, the
                                observer side over agents (no per-world barriers) then a thread per
                                agent for the partner side and the dynamics; 0 = one fused launch over
                                worlds.  Both give bit-identical gradients. */
  int32_t adjoint_recompute; /* states of a checkpoint segment recomputed by the backward pass
                                (GD_DIFFERENTIABLE): 1 (default) = one thread-per-agent launch per
                                segment from the objective rollout's record of its decisions (each
                                step's post-step flags, A bytes per step of episode_len, allocated
                                at create; without room for it, as 0);
                                0 = the step kernel, one launch per step.  Both give bit-identical
                                states, so bit-identical gradients. */
} gd_config;

typedef struct gd_scene_batch {
  int32_t num_worlds;
  const int32_t* agent_off;  /* [W+1], agent_off[0] = 0, non-decreasing */
  const int32_t* road_off;   /* [W+1], road_off[0] = 0, non-decreasing */
  const float *x, *y, *theta, *v;           /* [A] initial state */
  const float *length, *width;              /* [A] box extents, > 0 */
  const float *goal_x, *goal_y;             /* [A] */
  const uint8_t* agent_type;                /* [A] GD_AGENT_* */
  const float *road_x, *road_y;             /* [N] */
  const uint8_t* road_type;                 /* [N] GD_ROAD_* */
  const int32_t* road_poly;                 /* [N] polyline id; consecutive GD_ROAD_EDGE
                                               points of one polyline form a segment */
} gd_scene_batch;

typedef struct gd_info {
  int32_t num_worlds, num_agents, num_road, feat;   /* feat = F */
  int32_t max_agents_per_world, k_road, n_partners, episode_len;
  int64_t device_bytes;                             /* device memory owned by the env */
  int32_t block_size;                               /* threads per block of the batched step kernel in use */
  float road_cell;                                  /* road grid cell in use (m) */
  int32_t topk_strategy;                            /* road top-K method in use */
  int32_t lidar_rays;                               /* rays per agent (0 = LiDAR not enabled) */
  float lidar_fov;                                  /* rad */
  int32_t lidar_block_size;                         /* fused LiDAR kernel threads per block in use */
  int32_t lidar_road_tile;                          /* 1: it copies each world's road into shared memory */
  int32_t lidar_split;                              /* 1: step and LiDAR scan are two launches */
  int32_t road_tile;                                /* 1: the batched step kernel copies each world's road into
                                                       shared memory */
  int32_t obs_split;                                /* 1: step and radial observation are two launches */
  int32_t adjoint_split;                            /* 1: the step's adjoint is two launches (split form) */
  int32_t adjoint_road_tile;                        /* 1: the fused adjoint copies each world's road into
                                                       shared memory */
  int32_t objective_graph_kernels, objective_graph_other;  /* nodes of the captured gd_rollout_objective graph:
                                                              kernel launches, other nodes (copies, memsets);
                                                              0 while none is captured */
  int32_t backward_graph_kernels, backward_graph_other;    /* the same for gd_rollout_backward */
  int32_t adjoint_recompute;                                /* 1: the backward pass recomputes a segment in one
                                                              launch from the recorded decisions; 0: the step
                                                              kernel per step (see gd_config) */
} gd_info;

typedef struct gd_env gd_env;

/* Fill *cfg with the defaults listed above. */
void gd_default_config(gd_config* cfg);

/* Validate and upload a scene batch; build the static road grids.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which every
 * later call of this env runs.  Blocks until the upload is complete.
 * Errors: GD_ERR_INVALID_ARG (bad sizes, offsets, non-finite values),
 * GD_ERR_CAPACITY (a world above GD_MAX_AGENTS_PER_WORLD, K or P above the
 * limits), GD_ERR_OOM, GD_ERR_CUDA.  On error *out is NULL. */
gd_status gd_create(const gd_config* cfg, const gd_scene_batch* scene, void* cuda_stream, gd_env** out);

/* Synchronise the env's stream and free everything.  NULL is a no-op. */
gd_status gd_destroy(gd_env* env);

gd_status gd_get_info(const gd_env* env, gd_info* info);

/* Reset worlds to their initial snapshot (state, flags, episode step).
 * world_mask: device uint8 [W]; non-zero = reset; NULL = every world. */
gd_status gd_reset(gd_env* env, const uint8_t* world_mask);

/* One step of every world (see the header comment for the order).
 * actions: device float [A,2] = (acceleration m/s^2, steering rad).
 * reward: device float [A]; done: device uint8 [A] (1 = agent done after
 * this step); world_done: device uint8 [W] (1 = the world's episode ended).
 * Any output may be NULL.  Agents done before the step do not move, get
 * reward 0 and are invisible to the others. */
gd_status gd_step(gd_env* env, const float* actions, float* reward, uint8_t* done, uint8_t* world_done);

/* Observation of every agent after the last step (layout in the header
 * comment).  obs: device float [A,F], 16-byte aligned.  road_idx: device
 * int32 [A,K] local road indices of the slots (-1 = empty) or NULL;
 * partner_idx: device int32 [A,P] local agent indices or NULL. */
gd_status gd_observe(gd_env* env, float* obs, int32_t* road_idx, int32_t* partner_idx);

/* gd_step followed by gd_observe; with GD_BATCHED, two launches (obs_split = 1)
 * or one fused launch (obs_split = 0). */
gd_status gd_step_observe(gd_env* env, const float* actions, float* reward, uint8_t* done, uint8_t* world_done,
                          float* obs);

/* T = steps steps of gd_step_observe, replayed from a captured CUDA graph.
 * actions: device float [T,A,2]; obs: device float [A,F] (overwritten every
 * step) if obs_per_step == 0, else [T,A,F]; reward: float [T,A] or NULL;
 * done: uint8 [T,A] or NULL.  With GD_DIFFERENTIABLE the state is also
 * checkpointed every ckpt_every steps for gd_rollout_backward. */
gd_status gd_rollout(gd_env* env, int32_t steps, const float* actions, float* obs, int32_t obs_per_step,
                     float* reward, uint8_t* done);

/* LiDAR / view-cone observation of every agent after the last step
 * (Sec. 3.2 "Sensor modalities"; Fig. 1: 3000 rays over 360 degrees, or
 * over a 120-degree cone).  Requires lidar_rays > 0 at gd_create.  With
 * n = lidar_rays and fov = lidar_fov, ray k of agent i leaves the agent's
 * centre at angle
 *     theta_i + head[i] - fov/2 + (k + 1/2) fov / n
 * and stops at the first point at distance 0 <= t <= obs_radius that lies
 * in the closed box of another agent still in the scene (not done) or on a
 * road-edge segment (consecutive GD_ROAD_EDGE points of one polyline; lane
 * centre lines do not block rays).  The ray reports depth = t and class 1
 * (agent) or 2 (road edge), the agent at equal t; a ray that meets nothing
 * reports depth = obs_radius, class 0.  An agent inside another box sees
 * depth 0 on every ray.  Rows of done agents are all zero.  Depths are
 * float32 (the lowest mantissa bit may be cleared: one unit in the last
 * place).
 *   head:  device float [A] head rotation (rad, relative to the heading) or
 *          NULL = 0; 4-byte aligned
 *   depth: device float [A, n] (m); 4-byte aligned (16 for the fastest
 *          stores when n is a multiple of 4)
 *   cls:   device uint8 [A, n] or NULL
 * Errors: GD_ERR_STATE if the env has no LiDAR, GD_ERR_INVALID_ARG for NULL
 * or misaligned pointers. */
gd_status gd_observe_lidar(gd_env* env, const float* head, float* depth, uint8_t* cls);

/* gd_step followed by gd_observe_lidar; one fused launch when GD_BATCHED is
 * set.  Arguments as for gd_step and gd_observe_lidar. */
gd_status gd_step_observe_lidar(gd_env* env, const float* actions, const float* head, float* reward, uint8_t* done,
                                uint8_t* world_done, float* depth, uint8_t* cls);

/* T = steps steps of gd_step_observe_lidar (a captured CUDA graph when
 * GD_BATCHED is set).  actions: device float [T,A,2]; head: device float
 * [T,A] or NULL; depth / cls: [A,n] overwritten every step if
 * obs_per_step == 0, else [T,A,n] (cls may be NULL); reward: float [T,A]
 * or NULL; done: uint8 [T,A] or NULL. */
gd_status gd_rollout_lidar(gd_env* env, int32_t steps, const float* actions, const float* head, float* depth,
                           uint8_t* cls, int32_t obs_per_step, float* reward, uint8_t* done);

/* Episode statistics of the current state (the rates the paper reports:
 * goal reached, collision, off-road; Sec. 4): per world and in total, the
 * GD_STATS counts (in this order) of agents in the scene (not done),
 * controlled agents in the scene (not done, not GD_FLAG_STATIC), and agents
 * with GD_FLAG_GOAL, GD_FLAG_COLLIDED and GD_FLAG_OFFROAD set.
 *   per_world: device int32 [W, GD_STATS] or NULL
 *   totals:    device int64 [GD_STATS] or NULL (not both NULL)
 * Asynchronous. */
#define GD_STATS 5
gd_status gd_episode_stats(gd_env* env, int32_t* per_world, int64_t* totals);

/* Expert actions of trajectories under the env's dynamics model (Sec. 3.2
 * "Agent dynamics": actions computed from logged trajectories and replayed
 * to imitate them).  For each agent i and step t, from states s0 = state(t),
 * s1 = state(t+1):
 *   accel = (v1 - v0) / dt;  dtheta = theta1 - theta0 wrapped to [-pi, pi];
 *   GD_DYN_INVERTIBLE: steer = dtheta / (v0 dt + accel dt^2 / 2), 0 when that
 *     distance is <= 1e-6 m; replaying the actions reproduces the trajectory
 *     (the model is invertible);
 *   GD_DYN_BICYCLE: with k = dtheta L / (v-bar dt), v-bar = v0 + accel dt / 2,
 *     k clamped to +-1.99: steer = atan(k / sqrt(1 - k^2 / 4)), 0 when
 *     |v-bar dt| <= 1e-6 m; replaying matches heading and speed while no
 *     speed is clipped, not the positions (the model is not invertible).
 * L is each agent's length from the scene.  Agents' flags are not used.
 *   states:  device float [steps+1, A, 4] (x, y, theta, v), 16-byte aligned
 *   actions: device float [steps, A, 2] (accel, steer), 8-byte aligned
 * Asynchronous; errors: GD_ERR_INVALID_ARG (NULL, misaligned, steps < 0). */
gd_status gd_invert_actions(gd_env* env, int32_t steps, const float* states, float* actions);

/* gd_rollout with the per-step inputs and outputs in HOST memory (the end-
 * to-end call): actions_host [T,A,2] are copied in and reward_host [T,A] /
 * done_host [T,A] copied out in chunks of 8 steps on a second stream, so
 * that the copies overlap the steps; obs is device memory [A,F],
 * overwritten every step.  The copies and launches are one captured CUDA
 * graph (re-used while the pointers and steps are the same).  Host buffers
 * must be page-locked (cudaHostAlloc or registered); reward_host and
 * done_host may be NULL.  Asynchronous on the env's stream: the host buffers
 * must stay untouched until gd_sync.  Requires GD_BATCHED.  A device staging
 * of 13 bytes per agent-step is allocated on the first call.
 * Errors: GD_ERR_STATE without GD_BATCHED, GD_ERR_INVALID_ARG for NULL,
 * misaligned or pageable buffers. */
gd_status gd_rollout_host(gd_env* env, int32_t steps, const float* actions_host, float* obs, float* reward_host,
                          uint8_t* done_host);

/* Differentiable rollout (an extension; the paper has no gradient).  Runs
 * `steps` steps from the current state, like gd_rollout, and writes
 * the per-step objective terms
 *   ell[t,i] = sum_f obs_weight[f] * obs(t)[i,f] + reward_weight * r_s(t,i)
 * where obs(t) is the observation after step t and r_s = -(sqrt(d_goal^2 +
 * c^2) - c), c = smooth_c, for controlled agents in the scene at the start
 * of step t (0 otherwise).  The state is checkpointed every ckpt_every steps for
 * gd_rollout_backward; `actions` must stay unchanged until then.
 * Requires GD_DIFFERENTIABLE; steps <= episode_len.  With GD_BATCHED the
 * rollout (checkpoint copies and step launches) is one captured CUDA graph,
 * re-used while steps and the pointer and weight arguments are the same;
 * without it every launch is issued from the host.  Both give identical
 * results.
 *   actions: device float [T,A,2]; obs_weight: device float [F], 16-byte
 *   aligned; ell: device float [T,A]; obs: device float [A,F] overwritten
 *   every step, or NULL (an internal buffer is used). */
gd_status gd_rollout_objective(gd_env* env, int32_t steps, const float* actions, const float* obs_weight,
                               float reward_weight, float* ell, float* obs);

/* Gradient of  L = sum_{t,i} d_ell[t,i] * ell[t,i]  (d_ell = NULL: all ones)
 * for the last gd_rollout_objective, w.r.t. its actions and its initial
 * state.  Collision, goal, done, selection and clip decisions are held
 * constant.  Recomputes the states between checkpoints; the env's current
 * state is not changed.  obs_weight / reward_weight must be the values used
 * in the forward call.  With GD_BATCHED the whole backward pass (per
 * segment, last first: the checkpoint copy, the recomputed steps, the
 * adjoint of each step in reverse) is one captured CUDA graph with no
 * memset or copy node per step, re-used while the arguments are the same;
 * without it every launch is issued from the host.
 *   d_ell: device float [T,A] or NULL; d_actions: device float [T,A,2];
 *   d_state0: device float [A,4] or NULL. */
gd_status gd_rollout_backward(gd_env* env, const float* obs_weight, float reward_weight, const float* d_ell,
                              float* d_actions, float* d_state0);

/* Instrumentation (no counterpart in the paper): the same backward pass as
 * gd_rollout_backward, with the same arguments and results, but every launch
 * issued from the host with CUDA events around it.  Blocks until done; then
 * ms[k] holds the total milliseconds and launches[k] the number of launches
 * of kind k (GD_BWD_KINDS entries each, host memory):
 *   0 checkpoint copies (k_copy_snapshot), one per segment;
 *   1 recomputed states: one k_recompute launch per segment from the
 *     objective rollout's recorded decisions (gd_info.adjoint_recompute = 1),
 *     else the step kernel, out of place, one per step;
 *   2 the adjoint's observer side (split form: one launch per checkpoint
 *     segment, all its steps) or the whole fused adjoint (one per step);
 *   3 the split adjoint's per-agent part (partner side and dynamics of all
 *     the segment's steps, one launch per segment).
 * Per-launch averages are ms[k] / launches[k]. */
#define GD_BWD_KINDS 4
gd_status gd_time_backward(gd_env* env, const float* obs_weight, float reward_weight, const float* d_ell,
                           float* d_actions, float* d_state0, float* ms, int32_t* launches);

/* Instrumentation, as gd_time_backward: gd_rollout_objective (same arguments
 * and results; obs must not be NULL) with every launch issued from the host
 * under CUDA events.  Blocks.  Kinds (GD_OBJ_KINDS):
 *   0 checkpoint copies (k_copy_snapshot);
 *   1 step launches of the split form (the step kernel, writing r_s);
 *   2 observation launches of the split form (completing the objective
 *     terms), or the fused step + observation launches. */
#define GD_OBJ_KINDS 3
gd_status gd_time_objective(gd_env* env, int32_t steps, const float* actions, const float* obs_weight,
                            float reward_weight, float* ell, float* obs, float* ms, int32_t* launches);

/* Adjoint of one step about the CURRENT state and the given actions
 * (the step is not applied; requires GD_DIFFERENTIABLE): given
 * d_state_next [A,4] = dL/d(state after the step) (NULL = zero), the
 * gradient of L w.r.t. the observation after the step, d_obs [A,F] (or one
 * row obs_weight [F] for every agent; both NULL = no observation term), and
 * d_reward_s [A] = dL/d r_s (NULL = none), returns d_state [A,4] =
 * dL/d(state before the step) and d_actions [A,2].  All device pointers. */
gd_status gd_step_backward(gd_env* env, const float* actions, const float* d_state_next, const float* d_obs,
                           const float* obs_weight, const float* d_reward_s, float* d_state, float* d_actions);

/* State snapshot: state device float [A,4] = (x, y, theta, v), flags device
 * uint8 [A] (GD_FLAG_*), t device int32 [W] = steps into the episode.  Any
 * pointer may be NULL.  gd_set_state re-derives each world's episode-end
 * status from the flags and t. */
gd_status gd_get_state(gd_env* env, float* state, uint8_t* flags, int32_t* t);
gd_status gd_set_state(gd_env* env, const float* state, const uint8_t* flags, const int32_t* t);

/* Autotuner of the batched form: times the step + observation for
 * every road grid cell in {6, 8, 12} m, CTA size
 * in {128, 256, 512} threads, with and without the shared-memory road tile,
 * top-K strategy in {1 bucket rank, 2 bitonic sort when at most 256
 * points are in range}, and the split or fused observation (obs_split),
 * and keeps the fastest; with GD_DIFFERENTIABLE it
 * also times one adjoint launch with and without the road tile
 * (reported by gd_get_info).  With LiDAR enabled it then times the fused
 * step + LiDAR scan with 128, 256 and 384 threads per block, each with and
 * without the shared-memory road tile, and the split form (step, then a
 * scan over all agents), and keeps the fastest (a scratch of
 * A * lidar_rays * 5 bytes is held during the call).  Every combination gives the same results.
 * Each combination is timed over windows of 4 steps at three points of an
 * episode: the current state and the states 1 and 2 strides of zero-action
 * steps later (stride: episode_len / 3, at most 32 steps).  A scratch of
 * 3 * (33 A + 5 W) + 8 A bytes is held during the call.
 * Synchronises the env's stream; the simulation state is unchanged
 * afterwards.  A captured gd_rollout graph is dropped and re-captured on the
 * next call. */
gd_status gd_autotune(gd_env* env);

/* Failure-detection self-test (no counterpart in the paper): launches one
 * block that waits, bounded by about wait_us microseconds (1..1,000,000),
 * on a barrier phase nothing completes, and records the timeout in the
 * env's sticky error word exactly as the fused kernel's bounded copy waits
 * do; the next gd_sync returns GD_ERR_TIMEOUT.  No GPU fault is involved. */
gd_status gd_selftest_timeout(gd_env* env, int32_t wait_us);

/* Block until the env's stream is idle and report any sticky device error
 * (and clear it). */
gd_status gd_sync(gd_env* env);

const char* gd_last_error(const gd_env* env);

/* ---- polyline decimation at scene load --------------------------------------
 * Visvalingam-Whyatt decimation (Sec. 3.1: road polylines sampled every
 * 0.1 m are mostly straight; dropping low-importance points cuts them 10-15x
 * and speeds up the step).  For every polyline, the interior point of least
 * effective area (the triangle it spans with its two current neighbours;
 * ties: lower index) is eliminated while that area is below area_tol (m^2);
 * its neighbours' areas are recomputed with their new neighbours and raised
 * to the eliminated area if smaller.  End points are always kept.  Areas are
 * float32 in a fixed rounding order, so the result is reproducible.
 *   num_polylines P, num_points N (= poly_off[P])
 *   poly_off  device int32 [P+1], CSR: polyline p is points poly_off[p] ..
 *             poly_off[p+1]-1 (non-decreasing, poly_off[0] = 0)
 *   x, y      device float [N]
 *   keep      device uint8 [N] output: 1 = kept
 * Stateless: it needs no env.  A scratch of 20 bytes per point is taken
 * from the stream-ordered allocator for the call; one thread works through
 * each polyline.  Errors: GD_ERR_INVALID_ARG (negative sizes, NULL, bad
 * tolerance), GD_ERR_OOM; message in gd_last_error(NULL). */
gd_status gd_decimate(int32_t num_polylines, int32_t num_points, const int32_t* poly_off, const float* x,
                      const float* y, float area_tol, uint8_t* keep, void* cuda_stream);

/* The same decimation over a whole scene batch at load, before gd_create.
 * The polylines are the maximal runs of consecutive road points of one world
 * with one road_poly id (lane centre lines and road edges alike).  The road
 * arrays of `scene` (HOST memory, as for gd_create) are decimated on the
 * device and the kept points written, in their order, world by world, to the
 * caller's HOST arrays:
 *   keep           uint8 [N] (1 = kept; N = road_off[num_worlds]) or NULL
 *   road_off_out   int32 [num_worlds + 1], CSR offsets of the kept points
 *   road_x_out, road_y_out  float [N]; road_type_out uint8 [N];
 *   road_poly_out  int32 [N]  (the first *num_kept entries are written)
 *   num_kept       int32: points kept
 * The agent arrays are not read; a caller passes them on unchanged with the
 * new road arrays to gd_create (road indices then count the kept points).
 * Blocks until done (device buffers of about 13 bytes per point are taken
 * from the stream-ordered allocator for the call).  Errors:
 * GD_ERR_INVALID_ARG (NULL, bad offsets, bad tolerance), GD_ERR_OOM,
 * GD_ERR_CUDA; message in gd_last_error(NULL). */
gd_status gd_decimate_scene(const gd_scene_batch* scene, float area_tol, void* cuda_stream, uint8_t* keep,
                            int32_t* road_off_out, float* road_x_out, float* road_y_out, uint8_t* road_type_out,
                            int32_t* road_poly_out, int32_t* num_kept);

/* ---- allocation-free collision query ---------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: a program whose GPU memory is owned by
 * another pool allocator (cudaMalloc from this library would fail or escape
 * that pool's accounting), or a latency-critical loop that cannot take the
 * synchronisation cudaMalloc / cudaFree may cause.  gd_create allocates, so
 * such callers use this stateless call instead.
 *
 * Computes, for every agent, whether its box overlaps the box of another
 * active agent of the same world (the test behind GD_FLAG_COLLIDED of
 * gd_step), through a per-world uniform grid.
 *   agent_off  HOST int32 [num_worlds+1], CSR offsets (as in gd_scene_batch)
 *   state      device float [A,4] = (x, y, theta, v), 16-byte aligned
 *   extent     device float [A,2] = (length, width), 8-byte aligned
 *   active     device uint8 [A] (0 = not in the scene) or NULL = all active
 *   cell       grid cell in m; must be >= the largest box diagonal, or
 *              collisions between boxes more than one cell apart are missed
 *   collided   device uint8 [A] output: 1 = overlap, 0 = none or inactive
 * Working memory is one fixed array in the library (GD_NOALLOC_MAX_AGENTS
 * agents, GD_NOALLOC_MAX_WORLDS worlds; about 1.2 MB held on every GPU that
 * loads the library until the process exits).  Larger inputs return
 * GD_ERR_CAPACITY; bad arguments GD_ERR_INVALID_ARG; the text is in
 * gd_last_error(NULL).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture.  With lazy module loading (the CUDA default)
 * that first call also loads the library's device code on the device, and
 * the driver then takes the array's memory (about 1.2 MB): make the first
 * call at initialisation, before a pool allocator reserves the GPU's
 * memory.  No later call allocates.  Each call copies agent_off from host
 * memory to the array on the given stream, so a call is not capturable: on
 * a stream that is being captured into a CUDA graph it returns
 * GD_ERR_INVALID_ARG and enqueues nothing.  Every call reuses the same
 * array (nothing in it needs to start at zero: each call writes what it
 * reads), so calls that overlap on the GPU, e.g. on two streams, race. */
#define GD_NOALLOC_MAX_AGENTS 262144
#define GD_NOALLOC_MAX_WORLDS 16384
gd_status gd_collide_noalloc(int32_t num_worlds, const int32_t* agent_off, const float* state, const float* extent,
                             const uint8_t* active, float cell, uint8_t* collided, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GD_H */
