// Brute-force CPU oracle of the batched driving-simulator step.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
// CUDA library is checked against.  Only the test suite, the smoke check and
// the CPU-baseline leg of the benchmark may load it; the library never does.
// It shares no code, header, table or constant generator with the CUDA path.
//
// Every quantity follows the paper (GPUDrive, arXiv 2408.01584) or, where the
// paper is silent, the readings written next to the code:
//   * dynamics: kinematic bicycle model, App. B (the seven equations for
//     v-dot, v-bar, beta, x-dot, y-dot, theta-dot and the four update lines),
//     or the simplified invertible model of Sec. 3.2 "Agent dynamics" (a
//     double integrator along the heading whose yaw turns by the steering
//     curvature times the distance covered), and the expert-action inversion
//     of a trajectory under either model;
//   * collision: agents are convex boxes (Sec. 3.2 "Simulator sharp-edges",
//     "Convex objects only"); the paper's BVH (Sec. 3.1) only prunes pairs,
//     so the oracle tests every pair;
//   * off-road: cars and cyclists collide when they drive through a road
//     edge, pedestrians may cross (Sec. 3.2 "Termination conditions");
//   * reward 1 on reaching the goal within delta, else 0, with optional
//     collision penalties (Sec. 3.2 "Rewards");
//   * termination on goal, optionally on collision; removal after the goal
//     (Sec. 3.2 "Termination conditions");
//   * the "all nontrivial" initialisation (Sec. 3.2 "Simulator sharp-edges",
//     "Initialization modes"): only agents more than a set distance (2 m)
//     from their goal at the start are controlled; the others (parked cars)
//     stay where they are, visible to the rest;
//   * observation: every agent and road point within a fixed radius, in the
//     agent's relative frame (Sec. 3.2 "Sensor modalities"; 50 m in Fig. 1),
//     truncated to the K / P nearest;
//   * smooth goal reward (not in the paper): r_s = -(sqrt(d^2 + c^2) - c);
//   * polyline decimation at scene load (Sec. 3.1): the Visvalingam-Whyatt
//     algorithm (the paper's citation: repeated elimination of the point of
//     least effective area);
//   * LiDAR / view cone: rays cast from the agent over the other agents'
//     boxes and the road edges, in a full circle or a cone turned by a head
//     rotation (Sec. 3.2 "Sensor modalities"; 3000 rays, 360 or 120 degrees
//     in Fig. 1).
//
// Selection is a full std::sort of every candidate by (d^2, index); collision
// tests every pair and every road-edge segment; every LiDAR ray is tested
// against every box and every road-edge segment of its world.  T = double for parity,
// T = float to measure single-precision rounding.
//
// Parity pins live in the test suite (closed forms of App. B, polygon
// clipping, rigid-motion invariance, brute-force counts); nothing here is
// pinned against itself.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <set>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// flag bits of the per-agent status byte (same meaning as the library's)
constexpr uint8_t F_DONE = 1, F_GOAL = 2, F_COLLIDED = 4, F_OFFROAD = 8, F_STATIC = 16;
// configuration flag bits
constexpr uint32_t C_TERM_COLLISION = 1, C_TERM_OFFROAD = 2, C_AUTO_RESET = 4, C_NONTRIVIAL_INIT = 32;
constexpr uint8_t ROAD_EDGE = 1;
constexpr uint8_t PEDESTRIAN = 2;

struct Config {
  int k_road, n_partners, episode_len;
  double obs_radius, goal_radius, dt, v_max, collision_penalty, offroad_penalty, smooth_c;
  uint32_t flags;
  int dynamics;    // 0: kinematic bicycle (App. B); 1: simplified invertible model (Sec. 3.2)
  double nontrivial_dist;   // m: with C_NONTRIVIAL_INIT, agents this close to their goal are not controlled
};

template <typename T>
struct Box { T cx, cy, ca, sa, hl, hw; };   // centre, heading (cos, sin), half extents

template <typename T>
struct Env {
  Config cfg;
  int W = 0, A = 0, N = 0;
  std::vector<int32_t> agent_off, road_off;
  std::vector<T> x, y, th, v;                 // current state
  std::vector<T> x0, y0, th0, v0;             // initial snapshot (for reset)
  std::vector<T> len, wid, gx, gy;
  std::vector<uint8_t> type, flags, flags0;
  std::vector<T> rx, ry;
  std::vector<uint8_t> rtype;
  std::vector<int32_t> rpoly;
  std::vector<int32_t> t;                     // steps taken in the current episode
  std::vector<uint8_t> world_done;            // end-of-episode status of the last step
  // road-edge segments per world: pairs of consecutive ROAD_EDGE points of one polyline
  std::vector<std::vector<std::pair<int, int>>> segs;
};

template <typename T>
T clip(T a, T lo, T hi) { return a < lo ? lo : (a > hi ? hi : a); }

// ---- App. B: kinematic bicycle model, l_r = 0.5 L, explicit Euler ----------
template <typename T>
void bicycle_step(const Config& c, T L, T accel, T steer, T& x, T& y, T& th, T& v) {
  const T dt = (T)c.dt, vmax = (T)c.v_max;
  const T vdot = accel;                                               // v-dot = a
  const T vbar = clip<T>(v + (T)0.5 * vdot * dt, -vmax, vmax);        // mid-step speed
  const T beta = std::atan((T)0.5 * std::tan(steer));                 // atan(l_r tan(delta) / L)
  const T xdot = vbar * std::cos(th + beta);
  const T ydot = vbar * std::sin(th + beta);
  const T thdot = vbar * std::cos(beta) * std::tan(steer) / L;
  x = x + xdot * dt;                                                  // uses theta_t
  y = y + ydot * dt;
  th = th + thdot * dt;
  v = clip<T>(v + vdot * dt, -vmax, vmax);
}

// ---- Sec. 3.2 "Agent dynamics": the simplified invertible model ------------
// Readings where the paper is silent: the state is the same (x, y, theta, v)
// with v the signed speed along the heading; the position is a double
// integrator along the heading of the start of the step, so the distance
// covered is ds = v dt + a dt^2 / 2; the yaw changes by the steering
// command s times ds (s is a curvature, 1/m), which is the printed update
// theta + s (v dt + a dt^2 / 2); the speed is v + a dt, not clipped (a clip
// would make the model non-invertible).  The vehicle length plays no part.
template <typename T>
void invertible_step(const Config& c, T accel, T curv, T& x, T& y, T& th, T& v) {
  const T dt = (T)c.dt;
  const T ds = v * dt + (T)0.5 * accel * dt * dt;
  x = x + std::cos(th) * ds;
  y = y + std::sin(th) * ds;
  th = th + curv * ds;
  v = v + accel * dt;
}

template <typename T>
void dynamics_step(const Config& c, T L, T a, T steer, T& x, T& y, T& th, T& v) {
  if (c.dynamics == 1) invertible_step<T>(c, a, steer, x, y, th, v);
  else bicycle_step<T>(c, L, a, steer, x, y, th, v);
}

// Heading change wrapped to (-pi, pi].
template <typename T>
T wrap_angle(T d) {
  const T pi = (T)3.14159265358979323846;
  while (d > pi) d -= 2 * pi;
  while (d <= -pi) d += 2 * pi;
  return d;
}

// Expert actions of one step of a trajectory, state s0 -> s1 (x, y, theta, v).
// Both models: a = (v1 - v0) / dt.  Simplified model: s = dtheta / ds with
// ds = v0 dt + a dt^2 / 2 (0 when |ds| <= 1e-6 m: a vehicle that does not
// move has no defined curvature); replaying (a, s) reproduces theta, v and
// the positions exactly.  Kinematic bicycle: with v-bar = v0 + a dt / 2 (no
// clip) the yaw rate equation of App. B gives k = dtheta L / (v-bar dt) =
// cos(beta) tan(delta) = u / sqrt(1 + u^2 / 4), u = tan(delta), so
// u = k / sqrt(1 - k^2 / 4) for |k| < 2 (k clamped to +-1.99; delta = 0 when
// |v-bar dt| <= 1e-6 m); theta and v are matched, the positions then follow
// the slip angle, which is why this model is not fully invertible.
template <typename T>
void invert_step(const Config& c, T L, const T* s0, const T* s1, T& accel, T& steer) {
  const T dt = (T)c.dt;
  accel = (s1[3] - s0[3]) / dt;
  const T dth = wrap_angle(s1[2] - s0[2]);
  if (c.dynamics == 1) {
    const T ds = s0[3] * dt + (T)0.5 * accel * dt * dt;
    steer = std::fabs(ds) > (T)1e-6 ? dth / ds : (T)0;
  } else {
    const T vb = s0[3] + (T)0.5 * accel * dt;
    if (std::fabs(vb * dt) <= (T)1e-6) {
      steer = 0;
    } else {
      const T k = clip<T>(dth * L / (vb * dt), (T)-1.99, (T)1.99);
      steer = std::atan(k / std::sqrt(1 - k * k / 4));
    }
  }
}

// ---- separating-axis penetration -----------------------------------------
// Penetration of two intervals [a0,a1] and [b0,b1]: the smaller push that
// separates them; positive iff they overlap with positive depth.
template <typename T>
T interval_pen(T a0, T a1, T b0, T b1) { return std::min(a1 - b0, b1 - a0); }

template <typename T>
void project_box(const Box<T>& b, T ux, T uy, T& lo, T& hi) {
  const T c = b.cx * ux + b.cy * uy;
  const T r = b.hl * std::fabs(ux * b.ca + uy * b.sa) + b.hw * std::fabs(-ux * b.sa + uy * b.ca);
  lo = c - r;
  hi = c + r;
}

// Minimum over the four box axes of the penetration depth: > 0 iff the two
// oriented rectangles share interior points (touching is not a collision).
template <typename T>
T box_box_pen(const Box<T>& p, const Box<T>& q) {
  const T axes[4][2] = {{p.ca, p.sa}, {-p.sa, p.ca}, {q.ca, q.sa}, {-q.sa, q.ca}};
  T m = INFINITY;
  for (auto& u : axes) {
    T a0, a1, b0, b1;
    project_box(p, u[0], u[1], a0, a1);
    project_box(q, u[0], u[1], b0, b1);
    m = std::min(m, interval_pen(a0, a1, b0, b1));
  }
  return m;
}

// Same for a box and a segment: the two box axes plus the segment normal.
template <typename T>
T box_seg_pen(const Box<T>& p, T sx0, T sy0, T sx1, T sy1) {
  const T ex = sx1 - sx0, ey = sy1 - sy0;
  const T el = std::sqrt(ex * ex + ey * ey);
  T axes[3][2] = {{p.ca, p.sa}, {-p.sa, p.ca}, {0, 0}};
  int na = 2;
  if (el > 0) { axes[2][0] = -ey / el; axes[2][1] = ex / el; na = 3; }
  T m = INFINITY;
  for (int k = 0; k < na; ++k) {
    const T ux = axes[k][0], uy = axes[k][1];
    T a0, a1;
    project_box(p, ux, uy, a0, a1);
    const T s0 = sx0 * ux + sy0 * uy, s1 = sx1 * ux + sy1 * uy;
    m = std::min(m, interval_pen(a0, a1, std::min(s0, s1), std::max(s0, s1)));
  }
  return m;
}

template <typename T>
Box<T> agent_box(const Env<T>& e, int i) {
  return Box<T>{e.x[i], e.y[i], std::cos(e.th[i]), std::sin(e.th[i]), e.len[i] / 2, e.wid[i] / 2};
}

template <typename T>
void reset_world(Env<T>& e, int w) {
  for (int i = e.agent_off[w]; i < e.agent_off[w + 1]; ++i) {
    e.x[i] = e.x0[i]; e.y[i] = e.y0[i]; e.th[i] = e.th0[i]; e.v[i] = e.v0[i];
    e.flags[i] = e.flags0[i];
  }
  e.t[w] = 0;
  e.world_done[w] = 0;
}

// End of a world's episode: every controlled agent done (a world with no
// controlled agent only times out), or t = T.  Agents that are not
// controlled (F_STATIC) never end and do not hold the episode open.
template <typename T>
bool world_is_done(const Env<T>& e, int w) {
  const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
  int controlled = 0;
  bool all = true;
  for (int i = a0; i < a1; ++i) {
    if (e.flags[i] & F_STATIC) continue;
    ++controlled;
    all = all && (e.flags[i] & F_DONE);
  }
  return (controlled > 0 && all) || e.t[w] >= e.cfg.episode_len;
}

// Decisions of one step for world w after the dynamics have moved its active
// agents: collision, off-road, goal, reward, done, episode end.
template <typename T>
void decide_world(Env<T>& e, int w, const std::vector<uint8_t>& active, float* reward, uint8_t* done,
                  uint8_t* world_done, double* coll_margin, double* off_margin, double* goal_margin,
                  double* smooth_r) {
  const Config& c = e.cfg;
  const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
  for (int i = a0; i < a1; ++i) {
    if (!active[i - a0] || (e.flags[i] & F_STATIC)) {     // out of the scene, or not controlled
      if (reward) reward[i] = 0.f;
      if (coll_margin) coll_margin[i] = -INFINITY;
      if (off_margin) off_margin[i] = -INFINITY;
      if (goal_margin) goal_margin[i] = INFINITY;
      if (smooth_r) smooth_r[i] = 0.0;
      continue;
    }
    const Box<T> bi = agent_box(e, i);
    // agent/agent: any other agent active at the start of the step
    T best = -INFINITY;
    for (int j = a0; j < a1; ++j) {
      if (j == i || !active[j - a0]) continue;
      best = std::max(best, box_box_pen(bi, agent_box(e, j)));
    }
    const bool collided = best > 0;
    // agent/road edge, not for pedestrians
    T obest = -INFINITY;
    if (e.type[i] != PEDESTRIAN) {
      for (auto& s : e.segs[w]) {
        obest = std::max(obest, box_seg_pen(bi, e.rx[s.first], e.ry[s.first], e.rx[s.second], e.ry[s.second]));
      }
    }
    const bool offroad = obest > 0;
    const T dx = e.x[i] - e.gx[i], dy = e.y[i] - e.gy[i];
    const T dg = std::sqrt(dx * dx + dy * dy);
    const bool at_goal = dg <= (T)c.goal_radius;
    const bool first_goal = at_goal && !(e.flags[i] & F_GOAL);
    uint8_t f = e.flags[i] & (uint8_t)~(F_COLLIDED | F_OFFROAD);
    if (at_goal) f |= F_GOAL;
    if (collided) f |= F_COLLIDED;
    if (offroad) f |= F_OFFROAD;
    if ((f & F_GOAL) || (collided && (c.flags & C_TERM_COLLISION)) || (offroad && (c.flags & C_TERM_OFFROAD)))
      f |= F_DONE;
    e.flags[i] = f;
    if (reward)
      reward[i] = (float)((first_goal ? 1.0 : 0.0) - (collided ? c.collision_penalty : 0.0) -
                          (offroad ? c.offroad_penalty : 0.0));
    if (coll_margin) coll_margin[i] = (double)best;
    if (off_margin) off_margin[i] = (double)obest;
    if (goal_margin) goal_margin[i] = (double)dg - c.goal_radius;
    if (smooth_r) {
      const double sc = c.smooth_c;
      smooth_r[i] = -(std::sqrt((double)dx * dx + (double)dy * dy + sc * sc) - sc);
    }
  }
  e.t[w] += 1;
  e.world_done[w] = world_is_done(e, w) ? 1 : 0;
  if (done)
    for (int i = a0; i < a1; ++i) done[i] = (e.flags[i] & (F_DONE | F_STATIC)) ? 1 : 0;
  if (world_done) world_done[w] = e.world_done[w];
}

// One full step of every world.  If post_state is given (float [A,4]) the
// active agents take that state instead of running the dynamics: this lets a
// test evaluate the decisions on exactly the state another implementation
// produced.
template <typename T>
void step(Env<T>& e, const float* actions, const float* post_state, float* reward, uint8_t* done,
          uint8_t* world_done, double* cm, double* om, double* gm, double* sr) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int w = 0; w < e.W; ++w) {
    if ((e.cfg.flags & C_AUTO_RESET) && e.world_done[w]) reset_world(e, w);
    const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
    std::vector<uint8_t> active(a1 - a0);
    for (int i = a0; i < a1; ++i) {
      active[i - a0] = !(e.flags[i] & F_DONE);
      if (!active[i - a0] || (e.flags[i] & F_STATIC)) continue;   // done and uncontrolled agents do not move
      if (post_state) {
        e.x[i] = post_state[4 * i + 0]; e.y[i] = post_state[4 * i + 1];
        e.th[i] = post_state[4 * i + 2]; e.v[i] = post_state[4 * i + 3];
      } else {
        dynamics_step<T>(e.cfg, e.len[i], (T)actions[2 * i], (T)actions[2 * i + 1], e.x[i], e.y[i], e.th[i], e.v[i]);
      }
    }
    decide_world(e, w, active, reward, done, world_done, cm, om, gm, sr);
  }
}

// Ego-frame coordinates of point (px, py) seen from agent i: rotate the
// offset by -theta_i.
template <typename T>
void ego_frame(const Env<T>& e, int i, T px, T py, T& xr, T& yr) {
  const T c = std::cos(e.th[i]), s = std::sin(e.th[i]);
  const T dx = px - e.x[i], dy = py - e.y[i];
  xr = c * dx + s * dy;
  yr = -s * dx + c * dy;
}

template <typename T, typename O>
void road_feature(const Env<T>& e, int i, int jg, O* f) {
  T xr, yr;
  ego_frame(e, i, e.rx[jg], e.ry[jg], xr, yr);
  f[0] = (O)xr; f[1] = (O)yr; f[2] = (O)e.rtype[jg]; f[3] = 1;
}

template <typename T, typename O>
void partner_feature(const Env<T>& e, int i, int j, O* f) {
  T xr, yr;
  ego_frame(e, i, e.x[j], e.y[j], xr, yr);
  const T dth = e.th[j] - e.th[i];
  f[0] = (O)xr; f[1] = (O)yr; f[2] = (O)std::cos(dth); f[3] = (O)std::sin(dth);
  f[4] = (O)e.v[j]; f[5] = (O)e.len[j]; f[6] = (O)e.wid[j]; f[7] = 1;
}

// Observation row of every agent: ego[8], partners[P][8], road[K][4],
// written as O (float for the library's layout, double for derivatives).
template <typename T, typename O>
void observe(const Env<T>& e, O* obs, int32_t* road_idx, int32_t* partner_idx) {
  const int K = e.cfg.k_road, P = e.cfg.n_partners;
  const long F = 8 + 8L * P + 4L * K;
  const T R2 = (T)e.cfg.obs_radius * (T)e.cfg.obs_radius;
#pragma omp parallel for schedule(dynamic, 1)
  for (int w = 0; w < e.W; ++w) {
    const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
    const int r0 = e.road_off[w], r1 = e.road_off[w + 1];
    std::vector<std::pair<T, int>> cand;
    for (int i = a0; i < a1; ++i) {
      O* row = obs + (long)i * F;
      std::fill(row, row + F, (O)0);
      if (road_idx) std::fill(road_idx + (long)i * K, road_idx + (long)(i + 1) * K, -1);
      if (partner_idx) std::fill(partner_idx + (long)i * P, partner_idx + (long)(i + 1) * P, -1);
      row[5] = (e.flags[i] & F_COLLIDED) ? 1 : 0;
      row[6] = (e.flags[i] & F_OFFROAD) ? 1 : 0;
      row[7] = (e.flags[i] & F_GOAL) ? 1 : 0;
      if (e.flags[i] & F_DONE) continue;                  // removed from the scene
      T gxr, gyr;
      ego_frame(e, i, e.gx[i], e.gy[i], gxr, gyr);
      row[0] = (O)e.v[i]; row[1] = (O)e.len[i]; row[2] = (O)e.wid[i];
      row[3] = (O)gxr; row[4] = (O)gyr;
      // partners: every other agent still in the scene within the radius
      cand.clear();
      for (int j = a0; j < a1; ++j) {
        if (j == i || (e.flags[j] & F_DONE)) continue;
        const T dx = e.x[j] - e.x[i], dy = e.y[j] - e.y[i];
        const T d2 = dx * dx + dy * dy;
        if (d2 <= R2) cand.emplace_back(d2, j - a0);
      }
      std::sort(cand.begin(), cand.end());
      for (int k = 0; k < P && k < (int)cand.size(); ++k) {
        partner_feature(e, i, a0 + cand[k].second, row + 8 + 8 * k);
        if (partner_idx) partner_idx[(long)i * P + k] = cand[k].second;
      }
      // road points within the radius
      cand.clear();
      for (int j = r0; j < r1; ++j) {
        const T dx = e.rx[j] - e.x[i], dy = e.ry[j] - e.y[i];
        const T d2 = dx * dx + dy * dy;
        if (d2 <= R2) cand.emplace_back(d2, j - r0);
      }
      std::sort(cand.begin(), cand.end());
      for (int k = 0; k < K && k < (int)cand.size(); ++k) {
        road_feature(e, i, r0 + cand[k].second, row + 8 + 8 * P + 4 * k);
        if (road_idx) road_idx[(long)i * K + k] = cand[k].second;
      }
    }
  }
}

// ---- LiDAR / view cone (Sec. 3.2 "Sensor modalities") ---------------------
// Readings where the paper is silent:
//   * ray k of n leaves the agent's centre at angle
//       phi_k = theta + head - fov/2 + (k + 1/2) fov / n,
//     fov = 2 pi for the LiDAR, a smaller cone for the human-like view;
//     head is the head-rotation action (rad, relative to the heading);
//   * rays stop at the first point, 0 <= t <= R (the observation radius),
//     that lies in the closed box of another agent still in the scene or on
//     a road-edge segment (lane centre lines are markings, not obstacles);
//   * depth = that t and class 1 (agent) or 2 (road edge), agent first at
//     equal t; nothing met: depth R, class 0;  an agent that is done sees
//     nothing (depth 0, class 0).
// Per ray the oracle also reports how fragile the result is: a candidate
// whose hit/miss decision is within `band` metres of flipping (near a
// segment end, a box corner, t = 0 or t = R) at a distance not beyond the
// nearest hit, or an agent hit and an edge hit within `band` of each other,
// marks the ray fragile; sens = |d depth / d phi| of the nearest hit.

// Ray p + t u, 0 <= t <= R, against the closed box b (slab method in the
// box frame).  Returns true on a hit (t = 0 when p is inside); `tc` is the
// hit distance (or where the near-miss would hit), `margin` the metres by
// which the hit/miss decision could flip (hit: the smallest slack of its
// conditions; miss: the largest violation) and `sens` = |dt/dphi|.
template <typename T>
bool ray_box(T px, T py, T ux, T uy, T R, const Box<T>& b, T& tc, T& margin, T& sens) {
  const T dx = px - b.cx, dy = py - b.cy;
  const T o[2] = {b.ca * dx + b.sa * dy, -b.sa * dx + b.ca * dy};
  const T v[2] = {b.ca * ux + b.sa * uy, -b.sa * ux + b.ca * uy};
  const T h[2] = {b.hl, b.hw};
  T lo = -INFINITY, hi = INFINITY;
  int near_axis = -1;
  sens = 0;
  for (int a = 0; a < 2; ++a) {
    if (v[a] == 0) {
      if (std::fabs(o[a]) > h[a]) { tc = INFINITY; margin = std::fabs(o[a]) - h[a]; return false; }
      continue;
    }
    T t1 = (-h[a] - o[a]) / v[a], t2 = (h[a] - o[a]) / v[a];
    if (t1 > t2) std::swap(t1, t2);
    if (t1 > lo) { lo = t1; near_axis = a; }
    hi = std::min(hi, t2);
  }
  tc = std::max(lo, (T)0);
  const bool hit = lo <= hi && hi >= 0 && tc <= R;
  if (hit) {
    margin = std::min(hi - lo, R - tc);
    if (lo < 0) margin = std::min(margin, hi);
    if (lo > 0 && near_axis >= 0) sens = lo * std::fabs(v[1 - near_axis] / v[near_axis]);
  } else {
    margin = std::max(std::max(lo - hi, -hi), tc - R);
  }
  return hit;
}

// Ray p + t u, 0 <= t <= R, against the segment a-b: p + t u = a + s (b - a)
// by Cramer's rule; a hit needs 0 <= s <= 1.  Outputs as for ray_box.
template <typename T>
bool ray_seg(T px, T py, T ux, T uy, T R, T ax, T ay, T bx, T by, T& tc, T& margin, T& sens) {
  const T dx = bx - ax, dy = by - ay;
  const T wx = ax - px, wy = ay - py;
  const T den = ux * dy - uy * dx;
  if (den == 0) { tc = INFINITY; margin = INFINITY; sens = 0; return false; }
  const T t = (wx * dy - wy * dx) / den;
  const T s = (wx * uy - wy * ux) / den;
  const T len = std::sqrt(dx * dx + dy * dy);
  tc = t;
  sens = std::fabs(t * (ux * dx + uy * dy) / den);
  const bool hit = s >= 0 && s <= 1 && t >= 0 && t <= R;
  if (hit)
    margin = std::min(std::min(s * len, (1 - s) * len), std::min(t, R - t));
  else
    margin = std::max(std::max(-s * len, (s - 1) * len), std::max(-t, t - R));
  return hit;
}

template <typename T>
void lidar(const Env<T>& e, int n, double fov, const float* head, const int32_t* sel, int nsel, double band,
           double* depth, uint8_t* cls, uint8_t* fragile, double* sens_out) {
  const T R = (T)e.cfg.obs_radius;
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < nsel; ++q) {
    const int i = sel ? sel[q] : q;
    const int w = int(std::upper_bound(e.agent_off.begin(), e.agent_off.end(), i) - e.agent_off.begin()) - 1;
    const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
    for (int k = 0; k < n; ++k) {
      const long o = (long)q * n + k;
      depth[o] = 0; cls[o] = 0; fragile[o] = 0; sens_out[o] = 0;
    }
    if (e.flags[i] & F_DONE) continue;
    const T px = e.x[i], py = e.y[i];
    for (int k = 0; k < n; ++k) {
      const T phi = e.th[i] + (T)(head ? head[i] : 0.f) + (T)(-fov / 2 + (k + 0.5) * fov / n);
      const T ux = std::cos(phi), uy = std::sin(phi);
      // nearest hit of each class, then the winner
      T best[3] = {R, INFINITY, INFINITY}, bsens[3] = {0, 0, 0};
      T close_t = INFINITY;     // nearest candidate whose decision is within the band
      for (int j = a0; j < a1; ++j) {
        if (j == i || (e.flags[j] & F_DONE)) continue;
        T t, m, sn;
        const bool hit = ray_box(px, py, ux, uy, R, agent_box(e, j), t, m, sn);
        if (m < (T)band + (T)1e-6 * sn) close_t = std::min(close_t, t);
        if (hit && t < best[1]) { best[1] = t; bsens[1] = sn; }
      }
      for (auto& sg : e.segs[w]) {
        T t, m, sn;
        const bool hit = ray_seg(px, py, ux, uy, R, e.rx[sg.first], e.ry[sg.first], e.rx[sg.second],
                                 e.ry[sg.second], t, m, sn);
        if (m < (T)band + (T)1e-6 * sn) close_t = std::min(close_t, t);
        if (hit && t < best[2]) { best[2] = t; bsens[2] = sn; }
      }
      int c = 0;
      T d = R;
      if (best[1] <= R && best[1] <= best[2]) { c = 1; d = best[1]; }
      else if (best[2] <= R) { c = 2; d = best[2]; }
      bool frag = best[1] <= R && best[2] <= R && std::fabs(best[1] - best[2]) <= (T)band;
      frag = frag || close_t <= d + (T)band;
      const long o = (long)q * n + k;
      depth[o] = (double)d;
      cls[o] = (uint8_t)c;
      fragile[o] = frag ? 1 : 0;
      sens_out[o] = (double)bsens[c];
    }
  }
}

// ---- Sec. 3.1: Visvalingam-Whyatt polyline decimation ---------------------
// Effective area of point b between its current neighbours a and c (the
// triangle they span).  The paper fixes no precision, so the removal
// decisions are taken in the library kernel's: float32, in this operation
// order, with no fused multiply-add (the oracle is built with
// -ffp-contract=off).
static float vw_area(float ax, float ay, float bx, float by, float cx, float cy) {
  const float dx1 = bx - ax, dy1 = by - ay, dx2 = cx - ax, dy2 = cy - ay;
  const float p = dx1 * dy2;
  const float q = dx2 * dy1;
  return 0.5f * std::fabs(p - q);
}

// One polyline of n points.  End points are kept.  Repeatedly the interior
// point of least effective area (ties: lower index) is eliminated while that
// area is below tol; its neighbours' areas are recomputed with their new
// neighbours, and a recomputed area below the last eliminated one is raised
// to it (so the elimination order follows the areas monotonically).
static void vw_polyline(const float* x, const float* y, int n, float tol, uint8_t* keep) {
  for (int i = 0; i < n; ++i) keep[i] = 1;
  if (n < 3) return;
  std::vector<int> prev(n), next(n);
  std::vector<float> area(n, 0.f);
  std::set<std::pair<float, int>> queue;
  for (int i = 0; i < n; ++i) {
    prev[i] = i - 1;
    next[i] = i + 1;
  }
  for (int i = 1; i + 1 < n; ++i) {
    area[i] = vw_area(x[i - 1], y[i - 1], x[i], y[i], x[i + 1], y[i + 1]);
    queue.insert({area[i], i});
  }
  while (!queue.empty()) {
    const std::pair<float, int> m = *queue.begin();
    if (!(m.first < tol)) break;
    queue.erase(queue.begin());
    const int i = m.second;
    keep[i] = 0;
    const int a = prev[i], c = next[i];
    next[a] = c;
    prev[c] = a;
    for (int j : {a, c}) {
      if (j <= 0 || j >= n - 1) continue;
      queue.erase({area[j], j});
      area[j] = std::max(vw_area(x[prev[j]], y[prev[j]], x[j], y[j], x[next[j]], y[next[j]]), m.first);
      queue.insert({area[j], j});
    }
  }
}

struct Handle {
  int precision;   // 64 or 32
  void* env;
};

template <typename T>
Env<T>* make_env(const Config* cfg, int W, const int32_t* agent_off, const int32_t* road_off,
                 const float* x, const float* y, const float* th, const float* v, const float* len,
                 const float* wid, const float* gx, const float* gy, const uint8_t* atype,
                 const float* rx, const float* ry, const uint8_t* rtype, const int32_t* rpoly) {
  auto* e = new Env<T>();
  e->cfg = *cfg;
  e->W = W;
  e->agent_off.assign(agent_off, agent_off + W + 1);
  e->road_off.assign(road_off, road_off + W + 1);
  e->A = agent_off[W];
  e->N = road_off[W];
  auto cp = [](std::vector<T>& d, const float* s, int n) { d.resize(n); for (int i = 0; i < n; ++i) d[i] = (T)s[i]; };
  cp(e->x0, x, e->A); cp(e->y0, y, e->A); cp(e->th0, th, e->A); cp(e->v0, v, e->A);
  cp(e->len, len, e->A); cp(e->wid, wid, e->A); cp(e->gx, gx, e->A); cp(e->gy, gy, e->A);
  cp(e->rx, rx, e->N); cp(e->ry, ry, e->N);
  e->type.assign(atype, atype + e->A);
  e->rtype.assign(rtype, rtype + e->N);
  e->rpoly.assign(rpoly, rpoly + e->N);
  e->x = e->x0; e->y = e->y0; e->th = e->th0; e->v = e->v0;
  e->flags0.assign(e->A, 0);
  if (cfg->flags & C_NONTRIVIAL_INIT)
    for (int i = 0; i < e->A; ++i) {
      const double dx = (double)e->x0[i] - (double)e->gx[i], dy = (double)e->y0[i] - (double)e->gy[i];
      if (std::sqrt(dx * dx + dy * dy) <= cfg->nontrivial_dist) e->flags0[i] = F_STATIC;
    }
  e->flags = e->flags0;
  e->t.assign(W, 0);
  e->world_done.assign(W, 0);
  e->segs.resize(W);
  for (int w = 0; w < W; ++w)
    for (int j = road_off[w]; j + 1 < road_off[w + 1]; ++j)
      if (e->rtype[j] == ROAD_EDGE && e->rtype[j + 1] == ROAD_EDGE && e->rpoly[j] == e->rpoly[j + 1])
        e->segs[w].emplace_back(j, j + 1);
  return e;
}

template <typename T> Env<T>& env_of(Handle* h) { return *static_cast<Env<T>*>(h->env); }

}  // namespace

// ============================ C interface ==================================
// All arrays are host memory, rows in CSR agent order.  The oracle owns
// copies of everything it is given.
extern "C" {

typedef struct or_config {
  int32_t k_road, n_partners, episode_len;
  double obs_radius, goal_radius, dt, v_max, collision_penalty, offroad_penalty, smooth_c;
  uint32_t flags;
  int32_t dynamics;
  double nontrivial_dist;
} or_config;

void* or_create(const or_config* cfg, int precision, int32_t W, const int32_t* agent_off, const int32_t* road_off,
                const float* x, const float* y, const float* th, const float* v, const float* len,
                const float* wid, const float* gx, const float* gy, const uint8_t* atype, const float* rx,
                const float* ry, const uint8_t* rtype, const int32_t* rpoly) {
  Config c{cfg->k_road, cfg->n_partners, cfg->episode_len, cfg->obs_radius, cfg->goal_radius, cfg->dt,
           cfg->v_max, cfg->collision_penalty, cfg->offroad_penalty, cfg->smooth_c, cfg->flags, cfg->dynamics,
           cfg->nontrivial_dist};
  auto* h = new Handle{precision, nullptr};
  if (precision == 32)
    h->env = make_env<float>(&c, W, agent_off, road_off, x, y, th, v, len, wid, gx, gy, atype, rx, ry, rtype, rpoly);
  else
    h->env = make_env<double>(&c, W, agent_off, road_off, x, y, th, v, len, wid, gx, gy, atype, rx, ry, rtype, rpoly);
  return h;
}

void or_destroy(void* hv) {
  auto* h = static_cast<Handle*>(hv);
  if (h->precision == 32) delete &env_of<float>(h); else delete &env_of<double>(h);
  delete h;
}

#define OR_DISPATCH(h, ...) \
  do { if ((h)->precision == 32) { auto& e = env_of<float>(h); __VA_ARGS__; } \
       else { auto& e = env_of<double>(h); __VA_ARGS__; } } while (0)

// Reset the worlds whose mask byte is non-zero (all worlds if mask is NULL).
void or_reset(void* hv, const uint8_t* mask) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, for (int w = 0; w < e.W; ++w) if (!mask || mask[w]) reset_world(e, w));
}

// One step.  actions: float [A,2] (accel, steer).  Outputs may be NULL.
// Margins (double [A]): coll = max over partners of the box/box penetration,
// off = max over road-edge segments of the box/segment penetration (the flag
// is set iff the margin is > 0), goal = d_goal - delta; smooth = r_s.
void or_step(void* hv, const float* actions, float* reward, uint8_t* done, uint8_t* world_done,
             double* coll_margin, double* off_margin, double* goal_margin, double* smooth_r) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, step(e, actions, nullptr, reward, done, world_done, coll_margin, off_margin, goal_margin, smooth_r));
}

// The same step with the dynamics replaced by a given post-step state
// (float [A,4]); used to evaluate decisions on another implementation's state.
void or_step_post(void* hv, const float* post_state, float* reward, uint8_t* done, uint8_t* world_done,
                  double* coll_margin, double* off_margin, double* goal_margin, double* smooth_r) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, step(e, nullptr, post_state, reward, done, world_done, coll_margin, off_margin, goal_margin, smooth_r));
}

// Observation rows float [A, 8 + 8P + 4K]; index outputs int32 [A,K] / [A,P]
// (world-local indices, -1 padding) may be NULL.
void or_observe(void* hv, float* obs, int32_t* road_idx, int32_t* partner_idx) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, observe(e, obs, road_idx, partner_idx));
}

// The same rows in double precision (for derivative checks).
void or_observe64(void* hv, double* obs, int32_t* road_idx, int32_t* partner_idx) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, observe(e, obs, road_idx, partner_idx));
}

// Feature and exact distance of road point j (world-local) seen by agent i.
void or_road_point(void* hv, int32_t i, int32_t j, float* feat4, double* dist) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, {
    int w = int(std::upper_bound(e.agent_off.begin(), e.agent_off.end(), i) - e.agent_off.begin()) - 1;
    int jg = e.road_off[w] + j;
    road_feature(e, i, jg, feat4);
    double dx = (double)e.rx[jg] - (double)e.x[i], dy = (double)e.ry[jg] - (double)e.y[i];
    *dist = std::sqrt(dx * dx + dy * dy);
  });
}

// Feature and exact distance of agent j (world-local) seen by agent i.
void or_partner(void* hv, int32_t i, int32_t j, float* feat8, double* dist) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, {
    int w = int(std::upper_bound(e.agent_off.begin(), e.agent_off.end(), i) - e.agent_off.begin()) - 1;
    int jg = e.agent_off[w] + j;
    partner_feature(e, i, jg, feat8);
    double dx = (double)e.x[jg] - (double)e.x[i], dy = (double)e.y[jg] - (double)e.y[i];
    *dist = std::sqrt(dx * dx + dy * dy);
  });
}

// State as double [A,4] = (x, y, theta, v), flags [A], steps taken t [W],
// end-of-episode status [W].  Any output may be NULL.
void or_get_state(void* hv, double* state, uint8_t* flags, int32_t* t, uint8_t* world_done) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, {
    for (int i = 0; i < e.A; ++i) {
      if (state) { state[4 * i] = e.x[i]; state[4 * i + 1] = e.y[i]; state[4 * i + 2] = e.th[i]; state[4 * i + 3] = e.v[i]; }
      if (flags) flags[i] = e.flags[i];
    }
    for (int w = 0; w < e.W; ++w) { if (t) t[w] = e.t[w]; if (world_done) world_done[w] = e.world_done[w]; }
  });
}

// Overwrite the state from float [A,4] (and flags / t when given); the
// end-of-episode status is re-derived from them.
void or_set_state(void* hv, const float* state, const uint8_t* flags, const int32_t* t) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, {
    for (int i = 0; i < e.A; ++i) {
      if (state) { e.x[i] = state[4 * i]; e.y[i] = state[4 * i + 1]; e.th[i] = state[4 * i + 2]; e.v[i] = state[4 * i + 3]; }
      if (flags) e.flags[i] = flags[i];
    }
    if (t) for (int w = 0; w < e.W; ++w) e.t[w] = t[w];
    for (int w = 0; w < e.W; ++w) e.world_done[w] = world_is_done(e, w) ? 1 : 0;
  });
}

// Dynamics step (cfg->dynamics selects the model) of a flat array of
// independent agents (no world, no flags): state double [n,4] in place,
// actions double [n,2], length double [n].
void or_bicycle(const or_config* cfg, int64_t n, double* state, const double* actions, const double* length) {
  Config c{cfg->k_road, cfg->n_partners, cfg->episode_len, cfg->obs_radius, cfg->goal_radius, cfg->dt,
           cfg->v_max, cfg->collision_penalty, cfg->offroad_penalty, cfg->smooth_c, cfg->flags, cfg->dynamics,
           cfg->nontrivial_dist};
  for (int64_t i = 0; i < n; ++i)
    dynamics_step<double>(c, length[i], actions[2 * i], actions[2 * i + 1], state[4 * i], state[4 * i + 1],
                          state[4 * i + 2], state[4 * i + 3]);
}

// Expert actions of trajectories under cfg->dynamics (see invert_step):
// states double [steps+1, n, 4], length double [n]; actions double [steps, n, 2].
void or_invert(const or_config* cfg, int32_t steps, int64_t n, const double* states, const double* length,
               double* actions) {
  Config c{cfg->k_road, cfg->n_partners, cfg->episode_len, cfg->obs_radius, cfg->goal_radius, cfg->dt,
           cfg->v_max, cfg->collision_penalty, cfg->offroad_penalty, cfg->smooth_c, cfg->flags, cfg->dynamics,
           cfg->nontrivial_dist};
  for (int t = 0; t < steps; ++t)
    for (int64_t i = 0; i < n; ++i)
      invert_step<double>(c, length[i], states + ((int64_t)t * n + i) * 4, states + ((int64_t)(t + 1) * n + i) * 4,
                          actions[((int64_t)t * n + i) * 2], actions[((int64_t)t * n + i) * 2 + 1]);
}

// Penetration depth of two boxes (cx, cy, theta, length, width) and of a box
// and a segment; > 0 iff they share interior points.
double or_box_box(const double* p, const double* q) {
  Box<double> a{p[0], p[1], std::cos(p[2]), std::sin(p[2]), p[3] / 2, p[4] / 2};
  Box<double> b{q[0], q[1], std::cos(q[2]), std::sin(q[2]), q[3] / 2, q[4] / 2};
  return box_box_pen(a, b);
}

double or_box_seg(const double* p, const double* s) {
  Box<double> a{p[0], p[1], std::cos(p[2]), std::sin(p[2]), p[3] / 2, p[4] / 2};
  return box_seg_pen(a, s[0], s[1], s[2], s[3]);
}

// LiDAR / view-cone scan (readings above lidar()) of the agents listed in
// sel (int32 [nsel], global indices; NULL = all agents, nsel = A): n rays
// over fov radians about theta + head[i] (head float [A] or NULL = 0).
// Outputs [nsel, n]: depth double, cls uint8, fragile uint8, sens double.
void or_lidar(void* hv, int32_t n, double fov, const float* head, const int32_t* sel, int32_t nsel, double band,
              double* depth, uint8_t* cls, uint8_t* fragile, double* sens) {
  auto* h = static_cast<Handle*>(hv);
  OR_DISPATCH(h, lidar(e, n, fov, head, sel, nsel, band, depth, cls, fragile, sens));
}

// Visvalingam-Whyatt decimation of polylines (Sec. 3.1): polyline p is the
// points poly_off[p] .. poly_off[p+1]-1 of x, y (float32); keep (uint8 [N])
// gets 1 for the points that remain with area tolerance tol (m^2).
void or_decimate(int32_t num_polylines, const int32_t* poly_off, const float* x, const float* y, float tol,
                 uint8_t* keep) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int p = 0; p < num_polylines; ++p)
    vw_polyline(x + poly_off[p], y + poly_off[p], poly_off[p + 1] - poly_off[p], tol, keep + poly_off[p]);
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
